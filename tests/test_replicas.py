"""The multi-process path of bench.py on the CPU (gloo, world size 2), and
the bench line's host arithmetic.

A run does not shard: ``bench.py --gpus N`` runs N independent replicas, one
process per GPU.  What the replicas share is host logic: the barrier around
the timed steps, the slowest replica's time as the step time, and one JSON
line from rank 0.  These tests run that logic with the gloo backend on CPU
processes; nothing here needs a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.max_over_ranks(0.25 + 2.0 * rank, "cpu")
        with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
            f.write(repr(v))
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_slowest_replica(tmp_path):
    world = 2
    mp.start_processes(_max_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(world)]
    assert got == [2.25, 2.25]


def test_reference_arm_under_torchrun_prints_one_line_from_rank0():
    """torchrun with two ranks: rank 0 times the oracle and prints the line,
    rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--workload", "hilbert3d_n32",
           "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["config"]["workload"] == "hilbert3d_n32"
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["err"] <= 1e-10


def test_bench_host_helpers():
    """The bench line's host arithmetic: stored-residual GB/s over the median
    kernel time (none in the recompute form), and the dtype names."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench._stored_gbs({"stored_bytes": 0}, [1.0]) is None
    assert bench._stored_gbs({"stored_bytes": 2 * 10**9}, [3.0, 1.0, 2.0]) == 1000.0
    assert bench._dtype("fp64") == "f64" and bench._dtype("split") == "f32x2+f64"


def test_clock_samples_decoded():
    """nvidia-smi lines (SM clock, max clock, power, event-reason mask) become
    the line's clocks: median SM clock under load, the max clock, and the
    named reasons seen (idle left out)."""
    sys.path.insert(0, ROOT)
    import bench

    class FakeProc:
        stdout = ["2070, 2070, 900.1, 0x0000000000000000\n",
                  "1980, 2070, 1390.5, 0x0000000000000004\n",
                  "2070, 2070, 1100.0, 0x0000000000000001\n",
                  "garbage line\n",
                  "2055, 2070, 1200.0, 0x0000000000000020\n"]

        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler(0)
    c.proc = FakeProc()
    c._read()
    out = c.stop()
    assert out["samples"] == 4 and out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2062.5
    assert out["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
