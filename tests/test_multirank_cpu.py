"""The N > 1 path of bench.py on CPU: two gloo ranks build their own (different) potentials,
share nothing on the data path, and agree on the job time as the maximum over ranks."""

import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from lsp_inputs import make_workload
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_info()
    v = make_workload("helm2d_n32", seed=bench.rank_seed(r), n=16) if r == 0 else \
        make_workload("helm2d_n256", seed=bench.rank_seed(r), n=16)
    my_ms = 10.0 * (r + 1)  # a fake per-rank step time
    job_ms = bench.max_over_ranks(my_ms)
    value = bench.job_throughput(v.size, 5, ws, job_ms * 5)
    out[r] = (ws, r, float(v.sum()), job_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_seed_and_take_the_max_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2
    assert res[0][2] != res[1][2]                 # different potentials per rank
    assert res[0][3] == res[1][3] == 20.0         # both see the slowest rank's time
    # 2 ranks x 256 points x 5 steps over 100 ms
    assert np.isclose(res[0][4], 2 * 256 * 5 / 0.1)


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.rank_seed(0) is None and bench.rank_seed(3) == 1003
