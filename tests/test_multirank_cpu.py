"""Multi-process path of bench.py on CPU (gloo, world size 2): the reference arm runs on rank 0
only and the other rank exits cleanly; every rank joins the process group's barrier."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(600)
def test_bench_reference_arm_two_ranks_gloo():
    env = dict(os.environ)
    env.update(OMP_NUM_THREADS="2", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29531", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-n", "64"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["threads_busy"] > 0


def _shard_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import ddst_inputs as I
    from paper_2510_25991_gb300 import ddst as D
    specs = I.batch_specs(64)
    cost = [(s["n"] - 1) ** 2 for s in specs]
    owner, load = D.ddst_partition(cost, world)
    mine = [i for i, r in enumerate(owner) if r == rank]
    # every rank computes the same assignment without communication: gather and compare
    gathered = [None] * world
    dist.all_gather_object(gathered, (owner, mine))
    # the bench's timing reduction: the slowest rank's time (here its summed cost)
    t = torch.tensor([float(sum(cost[i] for i in mine))], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        with open(os.path.join(out_dir, "shards.json"), "w") as fh:
            json.dump({"gathered": gathered, "load": load, "max": float(t.item()), "cost": cost}, fh)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_batch_sharding_two_ranks_gloo(tmp_path):
    """The batch's sharding over ranks (ddst_partition, host only): two gloo ranks compute the
    same owner list independently, their shards are disjoint and cover the 64 problems, the
    loads are within 1% of each other, and the max-reduction of per-rank work equals the
    largest load."""
    import torch.multiprocessing as mp
    from paper_2510_25991_gb300 import build as B
    B.build()
    mp.start_processes(_shard_worker, args=(2, 29533, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    d = json.load(open(tmp_path / "shards.json"))
    (o0, m0), (o1, m1) = d["gathered"]
    assert o0 == o1
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    assert max(d["load"]) <= 1.01 * min(d["load"])
    assert d["max"] == max(d["load"])
    assert sum(d["load"]) == sum(d["cost"])
