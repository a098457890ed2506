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


def _lpt_worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    cfg, wseed, x, cu, sizes = bench.workload_inputs(rank, n_events=12, split="lpt", ws=ws)
    # the slowest rank sets the job's time; all ranks' events count once
    value, ms, ev = bench.job_throughput(ws, len(sizes), 20.0 - 5.0 * rank)
    out[rank] = (x, cu, sizes, value, ms, ev)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_lpt_split_of_one_batch():
    """Strong scaling: one batch split over two gloo ranks by the library's LPT rule;
    the ranks' events are disjoint, together they are the batch (the same elements),
    and the job's throughput is the batch over the slowest rank's time."""
    import synth
    from paper_2601_17554_b300 import shard_events
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_lpt_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    _, _, iseed, sizes = synth.workload("batch512")
    sizes = sizes[:12]
    shard, cost = shard_events(sizes, ws)
    x_all, cu_all = synth.gen_events(iseed, sizes)
    for r in range(ws):
        x, cu, sz, value, ms, ev = res[r]
        mine = np.nonzero(shard == r)[0]
        assert sz.tolist() == sizes[mine].tolist()
        expect = np.concatenate([x_all[cu_all[e]:cu_all[e + 1]] for e in mine])
        assert np.array_equal(x, expect)
        assert ms == 20.0 and ev == 12.0
        np.testing.assert_allclose(value, 12 / 0.020)
    assert sorted(np.concatenate([np.nonzero(shard == r)[0] for r in range(ws)]).tolist()) == list(range(12))
