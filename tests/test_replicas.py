"""The N > 1 host logic of bench.py on CPU: two gloo ranks.

The query of one string does not shard, so N GPUs run N independent
replicas.  What needs no GPU is checked here with world_size 2: rank 0
preps the workload and the other rank loads the same arrays, both replicas
compute the same answer (the oracle stands in for the device query), the
slowest rank's time is what every rank reports, and the whole-job value
counts the positions of all ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        ws, r, local = bench.dist_info()
        assert (ws, r, local) == (world, rank, rank)
        w = bench.load_workload("dna_64m", 6000, ws, r)
        res = oracle.lr_all_raw(w.rank, w.lcp)
        my_ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        ms = bench.max_over_ranks(my_ms)
        value = bench.whole_job_rate(ws, w.n, ms)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), sa=w.sa, lcp=w.lcp, offsets=res[2], starts=res[3],
                 ms=ms, value=value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    a = np.load(tmp_path / "rank0.npz")
    b = np.load(tmp_path / "rank1.npz")
    for k in ("sa", "lcp", "offsets", "starts"):
        assert np.array_equal(a[k], b[k]), k          # identical replicas, identical answers
    assert float(a["ms"]) == float(b["ms"]) == 15.0    # max over ranks
    assert float(a["value"]) == pytest.approx(2 * 6000 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 1000, 1.0) == pytest.approx(1e-3)
