"""The N-GPU benchmark path is replicas only: every rank advances its own chains, and
the job's rate is the units of all ranks over the slowest rank's timed region.  Its
host logic (replica streams, max over ranks, whole-job rate) runs here as two gloo
ranks on the CPU."""
import json
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    env = bench.dist_env()
    slowest_ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    rate = bench.job_throughput(ws, 5, slowest_ms / 1e3)
    out = {"env": env, "slowest_ms": slowest_ms, "rate": rate, "single": bench.replica_stream(rank, 1),
           "batch": bench.replica_stream(rank, 32)}
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"{rank}.json"), "w") as f:
        json.dump(out, f)


def test_two_gloo_ranks_aggregate_as_replicas(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"{r}.json")) for r in range(ws)]
    for r, o in enumerate(res):
        assert o["env"] == [ws, r, r]
        assert o["slowest_ms"] == 20.0                     # the slower rank's time on every rank
        assert o["rate"] == pytest.approx(2 * 5 / 0.020)   # units of both ranks over it
    # one chain per rank: same seed, distinct Philox chain ids; batches: distinct seeds
    assert res[0]["single"][0] == res[1]["single"][0] and res[0]["single"][1] != res[1]["single"][1]
    assert res[0]["batch"][0] != res[1]["batch"][0]
