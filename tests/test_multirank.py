"""Host logic of bench.py's multi-GPU launch (one process per GPU under torchrun), exercised with
two gloo ranks on the CPU: barriers around the timed region, the maximum of the ranks' times,
whole-job throughput from the units all ranks processed, rank 0 alone reporting, and the
reference arm's non-root ranks exiting without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    grp = bench.RankGroup("gloo")
    grp.barrier()
    t = grp.max_over_ranks(10.0 * rank + 5.0)  # this rank's "timed region" in ms
    grp.barrier()
    q.put((rank, grp.world, grp.is_root, t))
    grp.close()


def test_two_gloo_ranks_time_is_the_maximum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [True, False]
    assert all(o[3] == 15.0 for o in out)


def test_job_throughput_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    # 512 wavenumbers per rank and step, 2 ranks, 3 steps in 1.5 s -> 2048 solves/s
    assert bench.job_throughput(512, 2, 3, 1500.0) == pytest.approx(2048.0)
    assert bench.job_throughput(512, 1, 1, 1000.0) == pytest.approx(512.0)


def test_single_process_group_needs_no_distributed():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.get(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    for k in env:
        os.environ.pop(k, None)
    try:
        g = bench.RankGroup("gloo")
        assert g.world == 1 and g.is_root and g.dist is None
        assert g.max_over_ranks(3.5) == 3.5
        g.barrier()
        g.close()
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v


def test_reference_arm_non_root_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
