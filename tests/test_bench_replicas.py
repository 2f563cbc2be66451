"""The multi-GPU path of bench.py is replicas only: each rank solves its own
problem and the job time is the slowest rank's.  Its host logic runs here as
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        ms = bench.replica_time_max(10.0 * (rank + 1), torch.device("cpu"), ws)
        out[rank] = (ms, bench.replica_throughput(1e9, ms, ws))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # aggregate rate: both replicas' units over the slowest time
    assert res[0][1] == pytest.approx(2 * 1e9 / 0.020)


def test_single_rank_is_identity():
    import bench

    assert bench.replica_time_max(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.replica_throughput(10.0, 1000.0, 1) == pytest.approx(10.0)
