"""bench.py's multi-rank path on CPU: two gloo ranks, each timing its own
replica.  The whole-job figures are the slowest rank's time and the sum of
the ranks' units; every rank gets an independent image of the same shape
and PSF."""
import os
import sys
import tempfile

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, path, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"file://{path}", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate(dist, [3.5, 5.25][rank], [1000, 2500][rank], "cpu")
        w = bench.rank_workload("untiled-256", 10, rank)
        d = w.build(threshold=0.0)
        np.savez(os.path.join(out, f"r{rank}.npz"), ms=ms, units=units, seed=w.seed,
                 psf=d["psf"], dirty=d["dirty"])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_independent_replicas():
    with tempfile.TemporaryDirectory() as tmp:
        mp.start_processes(_worker, args=(2, os.path.join(tmp, "rdv"), tmp), nprocs=2, join=True,
                           start_method="spawn")
        r = [np.load(os.path.join(tmp, f"r{k}.npz")) for k in range(2)]
    for k in range(2):
        assert float(r[k]["ms"]) == 5.25          # max over ranks
        assert float(r[k]["units"]) == 3500.0     # sum over ranks
    import bench
    w0 = bench.rank_workload("untiled-256", 10, 0)
    assert int(r[0]["seed"]) == w0.seed           # rank 0 runs the single-GPU image
    assert int(r[1]["seed"]) != w0.seed
    assert np.array_equal(r[0]["psf"], r[1]["psf"])
    assert r[0]["dirty"].shape == r[1]["dirty"].shape
    assert not np.array_equal(r[0]["dirty"], r[1]["dirty"])


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, 7.0, 12) == (7.0, 12.0)
