"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
builds a distinct batch, the timed regions reduce to their maximum over
ranks, and the reference arm prints from rank 0 only."""
import json
import os
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.WORKLOADS["C2-batch"]["make"](n_inst=3, seed=bench.rank_seed(rank), nt=300)
    amp = w["eps"][:, -1, 0, 0].real
    t = bench.max_over_ranks([1.0 + rank, 5.0 - 3 * rank], dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, amp.tolist())
    if rank == 0:
        out.put((t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, amps = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == [2.0, 5.0]                       # max over ranks of each timed region
    assert amps[0][0] == amps[1][0] == 1.0       # instance 0 is C2 itself on every rank
    assert not np.allclose(amps[0][1:], amps[1][1:])   # the other instances differ per rank


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "C1",
                        "--steps", "1", "--warmup", "3",],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env["RANK"] = "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "C1",
                        "--steps", "1", "--warmup", "3",],
                       capture_output=True, text=True, env=env, timeout=300)
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
