"""Host-side logic of bench.py: the multi-rank aggregation (world size 2 over
gloo on CPU; every rank runs its own replica, the job value is all ranks'
work over the slowest rank's time) and the reference arm (the CPU oracle)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [1.5, 2.5][rank]
    m = bench.allreduce_max(dist, t)
    bench.barrier(dist)
    q.put((rank, m, bench.aggregate([10.0] * world, [1.5, 2.5])))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, agg in res:
        assert m == 2.5                      # slowest rank's time
        assert agg == pytest.approx(20.0 / 2.5)


def test_reference_arm_runs_the_oracle():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "grid2d-64", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Mnnz(G)/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    # the same metric string and workload description as the GPU arm prints
    sys.path.insert(0, ROOT)
    import bench
    assert line["metric"] == bench.METRIC
    assert line["config"]["workload"] == bench.WORKLOAD_DESC["grid2d-64"]
    assert line["pcg_iters"] > 0 and line["true_relres"] <= 1e-8 and line["cpu_baseline"]["tts_s"] > 0


def test_reference_arm_batch_sample():
    """The batch workload's reference arm factors a bounded sample of the 200
    systems (in order) with the oracle and says which."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "sddm-batch-200", "--steps", "1", "--warmup", "0", "--cpu-budget", "0.2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["systems"] == 200
    assert line["cpu_baseline"]["kind"] == "oracle" and "of 200 systems" in line["cpu_baseline"]["sample"]
