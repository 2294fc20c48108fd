"""The multi-GPU path's host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

The cells are independent, so ranks shard them with no collective on the data path; the
only collectives are the timing ones. Checked here: every rank gets the slowest rank's time
(max over ranks) after a barrier, the whole-job rate is all ranks' cells over that time,
each rank draws its own cells, and under torchrun the reference arm runs on rank 0 alone
(the other ranks exit 0 without work)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.rank_barrier(world)
    t = bench.max_over_ranks([0.7, 1.3][rank], world)
    q.put((rank, t, bench.job_rate(1000 * 10, world, t), bench.shard_seed(2003, rank)))
    bench.rank_barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.3, 1.3]
    assert all(abs(o[2] - 2 * 10000 / 1.3) < 1e-9 for o in out)
    assert out[0][3] != out[1][3]


def test_rank_shards_are_distinct_cells():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2312_05800_gb300 import synth
    m = synth.get_mech("c2")
    a = synth.states_profiles(m, 64, bench.shard_seed(2003, 0), ld=64)[0]
    b = synth.states_profiles(m, 64, bench.shard_seed(2003, 1), ld=64)[0]
    assert not np.any(a == b)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r1 = subprocess.run(cmd, env=dict(env, RANK="1", LOCAL_RANK="1"), capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, env=dict(env, RANK="0", LOCAL_RANK="0"), capture_output=True, text=True, timeout=600)
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
