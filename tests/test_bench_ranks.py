"""Host logic of bench.py for more than one rank (replicas, no data-path
collective): the per-step time is the maximum over ranks and the value counts
the bytes of every rank; on the oracle arm only rank 0 runs and prints.
Runs as two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.combine_ranks(1.0 + rank, world, 1_000_000)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(2.0)                       # slowest rank
        assert value == pytest.approx(world * 1.0 / 2e-3)     # 2 MB in 2 ms = 1000 MB/s


def test_combine_ranks_single():
    import bench
    ms, value = bench.combine_ranks(4.0, 1, 8_000_000)
    assert ms == 4.0 and value == pytest.approx(2000.0)


def test_reference_arm_only_rank0_prints():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("pred", ["mop", "learned"])
def test_reference_arm_line(pred):
    """Rank 0's reference arm (the oracle on the host) prints one JSON line
    with the keys the benchmark contract names; --pred learned runs the
    oracle with the bench's seeded net."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "vortex64", "--pred", pred, "--steps", "1", "--warmup", "0", "--cpu-slices", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MB/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["config"]["workload"] == "vortex64" and d["config"]["pred"] == pred
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["ratio"] > 1.0
