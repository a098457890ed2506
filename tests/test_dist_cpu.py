"""Multi-replica benchmark logic with two gloo ranks on CPU (no GPU).

Events are independent (no exchange step), so N GPUs run N replicas, each with
its own batch; the job's throughput is the events of all ranks over the slowest
rank's step time.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r processed 512 events in (10 + 5 r) ms
    value, ms, ev = bench.job_throughput(ws, 512, 10.0 + 5.0 * rank)
    cfg, wseed, x, cu, sizes = bench.workload_inputs(rank, n_events=8)
    out[rank] = (value, ms, ev, float(x[:, 8].sum()), int(sizes.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_distinct_batches():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        value, ms, ev, _, _ = res[r]
        assert ms == 15.0 and ev == 1024.0
        np.testing.assert_allclose(value, 1024 / 0.015)
    # weak scaling: each rank generates its own batch of the same distribution
    assert res[0][3] != res[1][3]
