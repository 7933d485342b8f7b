"""Host-side multi-rank logic of bench.py on the CPU (no GPU): the whole-job numbers of N
replicas (max over ranks of the step times, N steps' FLOPs per step) with two gloo ranks,
and the reference arm's rule that only rank 0 runs and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured 10 + r ms on the device and 20 + 3 r ms end to end
        res = bench.combine_ranks(10.0 + rank, 20.0 + 3 * rank, world, 2.0e9, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks(tmp_path):
    world = 2
    torch.multiprocessing.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    results = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert results[0] == results[1]  # every rank reports the same reduced numbers
    dev_ms, e2e_ms, value, e2e_value = results[0]
    assert dev_ms == 11.0 and e2e_ms == 23.0  # the slowest replica sets the step time
    assert value == pytest.approx(world * 2.0e9 / 11.0e-3 / 1e9)
    assert e2e_value == pytest.approx(world * 2.0e9 / 23.0e-3 / 1e9)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    dev_ms, e2e_ms, value, e2e_value = bench.combine_ranks(4.0, 5.0, 1, 1.0e9, "cpu")
    assert (dev_ms, e2e_ms) == (4.0, 5.0)
    assert value == pytest.approx(250.0) and e2e_value == pytest.approx(200.0)


def test_reference_arm_rank_nonzero_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
