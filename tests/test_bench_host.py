"""Host logic of bench.py that needs no GPU: which warm start each workload runs,
which workload the recorded PGS traffic belongs to, and how the CPU-baseline
sample is sized."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_warm_start_per_workload():
    # the large workload is specified with the learned warm start; the others run the prior frame
    assert bench.default_warm_start(5) == "learned"
    assert all(bench.default_warm_start(c) == "prior" for c in (1, 2, 3, 4))


def test_recorded_traffic_only_for_its_workload():
    rec = bench.PGS_TRAFFIC
    assert bench.pgs_traffic(3, 16384) is None
    assert bench.pgs_traffic(5, 65536) is None
    assert bench.pgs_traffic(rec["config"], 2 * rec["envs"]) is None
    got = bench.pgs_traffic(rec["config"], rec["envs"])
    assert got is None or got == rec["bytes"]


def test_oracle_legs_run_the_workloads_warm_start():
    o = bench.oracle_for(5, 4, "learned")
    assert o.params.warm_mode == 2
    assert bench.oracle_for(2, 4, "prior").params.warm_mode == 1
    assert bench.oracle_for(2, 4, "cold").params.warm_mode == 0


def test_cpu_sample_runs_whole_chunks_until_the_time_floor():
    rate, secs, steps = bench.oracle_run(2, 8, 2, 5, 2, min_s=0.3, max_s=5.0)
    assert steps % 5 == 0 and steps >= 5
    assert secs >= 0.3  # 8 small envs: the 5 s ceiling is never reached first
    assert rate == pytest.approx(8 * steps / secs)
    # a first chunk longer than the floor is the whole sample
    _, _, one = bench.oracle_run(2, 8, 0, 3, 2, min_s=0.0, max_s=5.0)
    assert one == 3


def test_training_seeds_are_disjoint_from_benchmark_and_held_out_seeds():
    # every rank's benchmark scenes (up to 8 x 65536 envs) and the warm-start study's
    # held-out scenes (offset 500000, 4096 envs) lie below the training offset
    assert bench.TRAIN_SEED_OFFSET > 8 * 65536 and bench.TRAIN_SEED_OFFSET > 500_000 + 4096
    assert np.all(np.arange(8) * 65536 + 65536 <= bench.TRAIN_SEED_OFFSET)
