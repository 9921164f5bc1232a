"""The multi-rank path on CPU (gloo, world size 2): each rank traces its own
shard of packages (package offsets rank * n under one random-number key), the
shards combine into one run of 2n packages, and bench.py's reductions take
the max of the timed spans and the sums of the work counters."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_1206_3710_gb300 import synth
        m = synth.tiny_clump()
        tree = oracle.Tree(m.tree)
        shard = bench.shard_params(rank, n)
        assert shard["job"] == 0
        res = oracle.trace(tree, m.sources, m.optics, n, seed=1002, packet_offset=shard["packet_offset"],
                           observers=m.observers, rr_wmin=1e-2, rr_p=0.5)
        ab = torch.from_numpy(res["absorbed"].copy())
        im = torch.from_numpy(res["images"].copy())
        bench.combine_shards(dist, world, ab, im)
        t, (cross, pk) = bench.reduce_over_ranks(dist, 10.0 + rank, [res["ledger"]["n_cross"], n], "cpu")
        one = oracle.trace(tree, m.sources, m.optics, world * n, seed=1002, observers=m.observers,
                           rr_wmin=1e-2, rr_p=0.5)
        # every rank holds the combined single run
        np.testing.assert_allclose(ab.numpy(), one["absorbed"], rtol=1e-12, atol=1e-15 * one["absorbed"].max())
        np.testing.assert_allclose(im.numpy(), one["images"], rtol=1e-12, atol=1e-15 * one["images"].max())
        assert one["images"].max() > 0
        if rank == 0:
            assert t == 10.0 + world - 1
            assert pk == world * n
            assert cross == one["ledger"]["n_cross"]
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo(orc):
    mp.spawn(_rank_main, args=(2, _free_port(), 1000), nprocs=2, join=True)
