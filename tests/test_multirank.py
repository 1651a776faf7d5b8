"""The benchmark's multi-rank path on CPU: two gloo ranks shard the video's
frames without overlap, agree on the slowest rank's step time, and report
the whole-job rate (the bench's only cross-rank exchange)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    frames = bench.rank_frames(rank, 250)
    my_ms = 100.0 + 25.0 * rank                     # rank 1 is the slower one
    ms_max = bench.max_over_ranks(my_ms, world)
    rate = bench.aggregate_rate(250, world, ms_max)
    q.put((rank, frames[0], frames[-1], ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, m0, v0), (r1, a1, b1, m1, v1) = res
    assert (a0, b0, a1, b1) == (0, 249, 250, 499)        # disjoint consecutive frames
    assert m0 == m1 == 125.0                            # both ranks see the slowest step
    assert v0 == v1 == pytest.approx(500 / 0.125)       # 500 pairs over 125 ms


def _bench(*args):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    return subprocess.run([sys.executable, os.path.join(root, "bench.py")] + list(args), capture_output=True,
                          text=True, timeout=300, env=env)


def test_bench_gpus_2_launches_two_ranks_through_torchrun():
    # bench.py --gpus 2 without a torchrun environment re-runs itself as two
    # ranks (torch.distributed.run, 127.0.0.1); the dry run does the ranks'
    # bookkeeping over gloo on CPU
    import json
    r = _bench("--gpus", "2", "--pairs", "3", "--rank-dry-run")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["n_gpus"] == 2 and line["frames"] == [[0, 1, 2], [3, 4, 5]]
    assert line["ms_per_step"] == 110.0 and line["value"] == pytest.approx(6 / 0.110)


def test_bench_gpus_n_needs_n_visible_gpus():
    import torch
    n = max(2, torch.cuda.device_count() + 1)
    r = _bench("--gpus", str(n), "--steps", "1")
    assert r.returncode == 2 and "needs %d visible GPUs" % n in r.stderr
