"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2).

Several GPUs run independent replicas of the job (realisations are
independent, no collective on the data path); the timing is the slowest
rank's and the rate counts every rank's units.
"""
import os
import socket

import pytest
import torch
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    ms = bench.max_over_ranks([100.0 + 50.0 * rank, 300.0 - 100.0 * rank], torch.device("cpu"))
    value = bench.job_throughput(1000, 3, dist.get_world_size(), ms[0])

    class A:
        warmup = 0
        steps = 1
    ref = bench.run_reference(A()) if rank == 1 else "skipped"
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(repr((ms, value, ref)))


def test_two_rank_timing_reduction_and_reference_arm(tmp_path):
    port = _free_port()
    tmp.spawn(_worker, args=(port, str(tmp_path)), nprocs=2, join=True)
    outs = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    for ms, value, _ in outs:
        assert ms == [150.0, 300.0]                   # the slowest rank's timings
        assert value == pytest.approx(1000 * 3 * 2 / 0.150)
    assert outs[1][2] is None                         # only rank 0 runs the reference arm


def test_single_process_reduction_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], torch.device("cpu")) == [1.5, 2.5]
    assert bench.job_throughput(10, 2, 1, 1000.0) == pytest.approx(20.0)


def test_gpus_flag_starts_one_rank_per_device_and_reduces():
    """`bench.py --gpus 2` without a launcher starts two ranks (torch.distributed.run,
    RANK / LOCAL_RANK / WORLD_SIZE per process); their host logic runs on gloo CPU
    ranks here and rank 0 alone prints the line, with the slowest rank's time."""
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                          "--steps", "3", "--dist-check"], capture_output=True, text=True,
                         timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    assert lines[0]["n_gpus"] == 2 and lines[0]["ms"] == 110.0
    assert lines[0]["value"] == pytest.approx(1000 * 3 * 2 / 0.110)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores (the paper
    ships no code) and prints one line with the reference keys."""
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["unit"] == "gap site-updates/s" and line["higher_is_better"] is True
