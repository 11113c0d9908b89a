"""Multi-rank host logic of bench.py, on two gloo ranks on the CPU.

The GPU leg runs one independent replica per rank (every rank digests,
deduplicates, restores and compares its own snapshot of the same shape); the
only cross-rank steps are the barriers and the reduction of the measured
times.  Here: the step time is the slowest rank's on every rank, the value
counts every replica's bytes, and in the reference arm only rank 0 works.
"""
import json
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, ms_by_rank, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(ms_by_rank[rank], world, "cpu")
        value = bench.whole_job_gbps(world, 1e9, ms)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_slowest_rank_and_value_counts_every_replica(tmp_path):
    world = 2
    ms_by_rank = [3.0, 5.0]
    mp.start_processes(_worker, args=(world, _free_port(), ms_by_rank, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == 5.0
        assert abs(r["value"] - world * 1e9 / 0.005 / 1e9) < 1e-9


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_gbps(1, 2e9, 1.0) == 2000.0


def test_reference_arm_works_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(seed=0, variant="full", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_clock_summary_prefers_samples_inside_the_timed_region():
    import bench
    cs = bench.ClockSampler(0)
    row = "0, {sm}, 2070, 900.00, 0x0, {hw}, Not Active, Not Active, {cap}"
    cs.lines = [(9.5, row.format(sm=1000, hw="Not Active", cap="Not Active")),     # before: idle, lower clock
                (10.1, row.format(sm=2070, hw="Not Active", cap="Active")),
                (10.3, row.format(sm=2050, hw="Not Active", cap="Not Active")),
                (10.5, row.format(sm=2070, hw="Not Active", cap="Not Active")),
                (11.2, row.format(sm=1000, hw="Active", cap="Not Active"))]        # after
    s = cs.summary(10.0, 11.0)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s = cs.summary(10.0, 10.2)                 # one sample inside: the neighbours within 0.25 s count too
    assert s["samples"] == 2 and s["sm_mhz"] == 2060.0
