"""The multi-rank logic of bench.py on the CPU: two gloo ranks (world size 2) agree on the slowest
rank's time and on the whole-job throughput, and the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(torch, dist, times[rank])
        assert t == max(times), (rank, t)
        cells, steps = 256 * 192 * 256, 50
        v = bench.job_throughput(world, cells, steps, t)
        assert v == world * cells * steps / max(times)
        # every rank computes the same value, as rank 0 reports it
        got = [None] * world
        dist.all_gather_object(got, v)
        assert len(set(got)) == 1
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    mp.start_processes(_worker, args=(2, _free_port(), [0.75, 1.25]), nprocs=2, join=True, start_method="spawn")


def test_single_process_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 0.5) == 0.5
    assert bench.job_throughput(1, 10, 4, 2.0) == 20.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    """The reference arm (the oracle timed on the host cores) prints one JSON line with the
    contract's keys, the same metric, unit and workload as the CUDA arm, and e2e equal to its
    own value with no host-device bytes."""
    import json
    env = dict(os.environ, RANK="0", LOCAL_RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert key in d, key
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["steps"] == 1
    assert d["warmup"] == 3  # the bench takes at least three warm-up steps whatever is asked
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["config"]["workload"] == "turbulent_channel_256x192x256_fp64"
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["cpu"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["gpu_launches"] == 0
