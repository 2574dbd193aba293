"""Host logic of bench.py on the CPU: the multi-rank reduction over two
gloo ranks, the parsing of the clock samples, and the reference arm's
ranks other than 0 exiting without work."""
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest

import bench

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: timings 10 + r and 5 - r ms, counts 100 (r + 1) and 7
        maxes, sums = bench.reduce_over_ranks(dist, "cpu", [10.0 + rank, 5.0 - rank],
                                              [100 * (rank + 1), 7])
        Path(out_dir, f"r{rank}.txt").write_text(repr((maxes, sums)))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks(tmp_path):
    """Every rank gets the slowest rank's times and the sum of all ranks'
    counts."""
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        maxes, sums = eval(Path(tmp_path, f"r{r}.txt").read_text())
        assert maxes == [11.0, 5.0]
        assert sums == [300.0, 14.0]


def test_reduce_single_process_is_identity():
    assert bench.reduce_over_ranks(None, "cpu", [3, 4.5], [216000]) == ([3.0, 4.5], [216000.0])


def test_clock_summary():
    """Median SM clock, the largest max clock, the reasons seen active in any
    sample; rows that are not samples are skipped."""
    def row(sm, mx, power_cap="Not Active", hw="Not Active"):
        return f"0, {sm}, {mx}, 812.5, 0x0000000000000004, {hw}, Not Active, Not Active, {power_cap}\n"
    lines = [row(2070, 2070), row(1980, 2070, power_cap="Active"), row(2070, 2070),
             "garbage\n", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active\n"]
    got = bench.clock_summary(lines)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    got = bench.clock_summary([row(1500, 2070, hw="Active"), row(1600, 2070)])
    assert got["sm_mhz"] == 1550.0 and got["reasons"] == ["hw_slowdown"]
    assert bench.clock_summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                                       "samples": 0}


@pytest.mark.parametrize("rank", [1, 3])
def test_reference_arm_other_ranks_exit_without_work(rank):
    """Under a 4-rank launch only rank 0 runs the oracle and prints; the
    others exit 0 at once and print nothing."""
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="4")
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                          "--gpus", "4", "--steps", "3", "--warmup", "3"],
                         capture_output=True, text=True, env=env, cwd=str(ROOT), timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_cpu_baseline_entry_records_the_host():
    """The oracle leg's entry: element applications per second over the
    sample, one thread, the host's core count and CPU model."""
    e = bench.cpu_baseline_entry({"times": [1.0, 3.0], "kv": [40, 40], "n_elem": 216000}, 40)
    assert e["value"] == 216000 * 80 / 4.0 / 1e9
    assert e["cores"] == 1 and e["kind"] == "oracle"
    assert isinstance(e["host_cores"], int) and e["host_cores"] >= 1
    assert isinstance(e["cpu_model"], str) and e["cpu_model"]
