"""bench.py's whole-job rate over ranks, on two gloo ranks on the CPU: the job's time is the
slowest rank's (all-reduce MAX), and the rate counts every rank's units.  Under torchrun
bench.py runs one independent replica per GPU and aggregates exactly this way."""
import json
import os
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, outdir: str):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    rate, ms = bench.job_rate(100.0 * (rank + 1), 21 * 10, world, dist, "cpu")
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as fh:
        json.dump({"rate": rate, "ms": ms}, fh)
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["ms"] == 200.0                        # rank 1's 200 ms on every rank
        assert abs(got["rate"] - world * 210 / 0.2) < 1e-9


def test_job_rate_single_rank():
    import bench

    rate, ms = bench.job_rate(250.0, 105, 1)
    assert ms == 250.0 and abs(rate - 420.0) < 1e-12
