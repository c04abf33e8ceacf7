"""The multi-process (N > 1) host logic of bench.py on CPU with gloo,
world size 2: rendezvous on 127.0.0.1, the barrier, the maximum of the
per-rank times, the replica throughput, and the reference arm under
torchrun (rank 0 alone runs and prints; the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world, backend="gloo")
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 + 5.0 * r, w)     # per-rank "times"
    bench.barrier(w)
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as fh:
        json.dump({"rank": r, "world": w, "local": local, "max": slowest}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert [d["rank"] for d in res] == [0, 1]
    assert all(d["world"] == 2 and d["max"] == 15.0 for d in res)


def test_replica_throughput_counts_every_rank_over_the_slowest_time():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 1e6 nodes x 10 steps in 0.5 s (the slowest rank)
    assert bench.replica_mlups(2, 1_000_000, 10, 0.5) == pytest.approx(40.0)
    assert bench.replica_mlups(1, 1_000_000, 10, 0.5) == pytest.approx(20.0)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 3
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle"
