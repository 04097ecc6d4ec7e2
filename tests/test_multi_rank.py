"""The N > 1 path of bench.py on CPU: max-over-ranks timing, the whole-job
rate of replicas and of sharded runs, the instance shares of the batched
workload, on a world-size-2 gloo process group where ranks are involved; the
reference arm's rank 1 exits without work or output."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # ranks finish their timed steps at different times; everyone must see
    # the slowest one
    ms = [1200.0, 1500.0][rank]
    mx = bench.max_over_ranks(ms, dist)
    rate = bench.whole_job_rate(3, world, mx)
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"max": mx, "rate": rate}, f)
    dist.destroy_process_group()


def test_replica_timing_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert res[0]["max"] == res[1]["max"] == 1500.0
    # 3 units per rank, 2 ranks, over the slowest rank's 1.5 s
    assert res[0]["rate"] == pytest.approx(4.0)


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(2, 1, 500.0) == pytest.approx(4.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_sharded_rate_and_instance_shares():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2512_01257_gb300 import build, rafeast as R
    if not os.path.exists(R.LIB_PATH):
        build.build()
    # one solve shared by the ranks in 250 ms: 4 solves/s whatever the N
    assert bench.sharded_rate(1, 250.0) == pytest.approx(4.0)
    costs = [int(c) for c in (np.random.default_rng(3).integers(1, 10**6, 64))]
    assert bench.my_instances(costs, 1, 0) == list(range(64))
    for world in (2, 3, 8):
        shares = [bench.my_instances(costs, world, r, R) for r in range(world)]
        # every problem solved once, by one rank
        assert sorted(t for s in shares for t in s) == list(range(64))
        loads = [sum(costs[t] for t in s) for s in shares]
        assert max(loads) <= sum(costs) / world + max(costs)
