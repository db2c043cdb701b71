"""Host logic of bench.py under several ranks, on the CPU (gloo, world size 2):
the replicas' times reduce to their maximum, and the reference arm runs on
rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # each replica reports its own time; every rank sees the slowest
        got = bench.max_over_ranks(10.0 + 7.5 * rank, world, "cpu")
        got2 = bench.max_over_ranks(3.0 - rank, world, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{got!r} {got2!r}\n")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        got, got2 = map(float, (tmp_path / f"rank{r}.txt").read_text().split())
        assert got == 17.5 and got2 == 3.0


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(4.25, 1, "cpu") == 4.25


def test_reference_arm_other_ranks_exit_quietly(repo_root):
    # under torchrun only rank 0 runs the CPU oracle and prints; rank 1 exits 0
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(repo_root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_dist_setup_reads_the_environment(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_setup() == (4, 3, 1)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k)
    assert bench.dist_setup() == (1, 0, 0)


def test_batch_shard_covers_every_mesh_once_and_balances():
    import bench
    import synth
    sizes = [m.n for m, _ in synth.batch(count=64)]
    for world in (1, 2, 3, 4, 8):
        parts = bench.batch_shard(sizes, world)
        assert len(parts) == world
        flat = sorted(i for part in parts for i in part)
        assert flat == list(range(64))
        loads = [sum(sizes[i] for i in part) for part in parts]
        # greedy largest-first: no rank carries more than the mean plus the largest mesh
        assert max(loads) <= sum(sizes) / world + max(sizes)
        assert parts == bench.batch_shard(sizes, world)        # deterministic
    parts = bench.batch_shard([5, 3], 4)                       # more ranks than meshes
    assert parts == [[0], [1], [], []]
