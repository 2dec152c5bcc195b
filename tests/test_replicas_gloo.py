"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the step
has no collective ("replicas only"), so N ranks each advance a replica; the
job's time is the slowest rank's and its throughput counts every replica.
The reference arm prints from rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {"max": bench.max_over_ranks(10.0 + 5.0 * rank)}
    res["value"] = bench.job_throughput(1000, world, res["max"])
    dist.barrier()

    class Args:
        steps, warmup = 1, 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(Args())
    res["printed"] = buf.getvalue()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_replica_timing_and_reference_arm_on_two_ranks(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    assert r[0]["max"] == r[1]["max"] == 15.0          # slowest rank's time on every rank
    assert r[0]["value"] == 1000 * 2 / 15e-3            # all replicas' cells / job time
    assert r[1]["printed"] == ""                        # reference arm: rank 0 alone prints
    line = json.loads(r[0]["printed"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
