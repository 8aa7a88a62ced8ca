"""Multi-rank source sharding on CPU: two gloo ranks each compute their
shard (with the oracle standing in for the GPU) and reduce in rank order."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_0809_1906_gb300 import graphs as G
from paper_0809_1906_gb300.sharding import shard_sources


def test_shards_partition_the_sources():
    src = np.arange(1000, dtype=np.int32)
    for world in (1, 2, 3, 8):
        parts = [shard_sources(src, r, world, 64) for r in range(world)]
        allv = np.sort(np.concatenate(parts))
        assert np.array_equal(allv, src)
        sizes = [p.size for p in parts]
        assert max(sizes) - min(sizes) <= 64


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_0809_1906_gb300.sharding import reduce_partials
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = G.er_hamiltonian(400, 1500, 21)
    mine = shard_sources(np.arange(g.n, dtype=np.int32), rank, world, 64)
    part = oracle.bc(g, mine, threads=1)["bc"]
    full = reduce_partials(part)
    import torch
    from paper_0809_1906_gb300.sharding import reduce_partials_device
    again = reduce_partials_device(torch.from_numpy(part)).numpy()
    assert np.array_equal(full, again)  # both sum the gathered vectors in rank order
    q.put((rank, full))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_two_ranks_sum_equals_single_run(world):
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = G.er_hamiltonian(400, 1500, 21)
    ref = oracle.bc(g, threads=1)["bc"]
    for r in range(world):
        assert np.allclose(res[r], ref, rtol=1e-12, atol=1e-9)
    assert np.array_equal(res[0], res[1])
