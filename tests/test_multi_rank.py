"""The multi-rank bench path on CPU: two gloo ranks exercise the helpers bench.py uses under
torchrun (rank environment, barrier, max-over-ranks timing, whole-job rate), and the
reference arm's rule that only rank 0 works. The count itself has no exchange step (every
rank counts its own replica), so nothing else crosses ranks.
"""

from __future__ import annotations

import json
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


def _rank_main(rank: int, world: int, port: int, out_dir: str, times: list) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        bench.rank_barrier(dist)
        ms = bench.max_over_ranks(times[r], dist, "cpu")
        rate = bench.whole_job_rate(w, 1_000.0, 4, ms)
        bench.rank_barrier(dist)
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump({"env": [w, r, local], "ms": ms, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    times = [12.5, 40.0]
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path), times), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, g in enumerate(got):
        assert g["env"] == [2, r, r]
        assert g["ms"] == max(times)                 # every rank sees the slowest rank's time
        # 2 ranks x 1,000 units x 4 steps in 40 ms
        assert g["rate"] == pytest.approx(2 * 1_000 * 4 / 0.040)


def test_single_process_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    bench.rank_barrier(None)
    assert bench.whole_job_rate(1, 500.0, 2, 1_000.0) == pytest.approx(1_000.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""                    # rank 0 alone prints the line
