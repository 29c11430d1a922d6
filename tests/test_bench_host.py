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


def test_timed_window_starts_at_step_60_whatever_the_warmup():
    # the default K = 20 times physics steps 60-360 of the headline workload (300 steps
    # after 60); workload 5 steps one target-refresh period per benchmark step
    args = bench.parse([])
    assert bench.timed_window(args.warmup, args.steps) == (60, 360)
    assert bench.timed_window(15, 20, 3) == (60, 360)
    assert bench.timed_window(5, 20, 5) == (60, 140)
    assert bench.timed_window(40, 1) == (60, 75)
    for cfg in (2, 3, 5):
        assert bench.WINDOW_START % bench.step_physics(cfg) == 0


def test_pgs_bytes_counts_every_item_class():
    t = {"n_contacts": 3, "n_pool_slots": 2, "n_limit_rows": 1, "n_envs": 5}
    B = bench.PGS_BYTES
    assert bench.pgs_bytes(t, 7, 11) == 7 * B["object"] + 11 * B["joint"] + 3 * B["contact"] + \
        2 * B["pool_slot"] + B["limit_row"] + 5 * B["env"]


def test_merged_cache_keeps_prior_entries_for_matched_contacts_only():
    """The ideal-start cache of the warm-start bounds: a contact of the step that matches
    a prior-frame entry (same key, point within the match distance) keeps the prior
    impulse; a new contact (new key, or a key whose point moved too far) gets the step's
    converged impulse; counts and keys are the step's."""
    C = 4
    S = {"cache_count": np.array([2, 1], np.int32),
         "cache_key": np.zeros((2 * C, 3), np.int32), "cache_p": np.zeros((2 * C, 3), np.float32),
         "cache_lambda": np.zeros((2 * C, 4), np.float32)}
    S["cache_key"][0:2] = [[0, 5, 1], [1, 5, 0]]
    S["cache_lambda"][0:2] = [[1, 0, 0, 0], [2, 0, 0, 0]]
    S["cache_key"][C] = [0, 3, 7]
    S["cache_p"][C] = [0.5, 0, 0]
    S["cache_lambda"][C] = [3, 0, 0, 0]
    post = {"cache_count": np.array([3, 1], np.int32),
            "cache_key": np.zeros((2 * C, 3), np.int32), "cache_p": np.zeros((2 * C, 3), np.float32),
            "cache_lambda": np.zeros((2 * C, 4), np.float32)}
    post["cache_key"][0:3] = [[0, 5, 1], [0, 6, 0], [1, 5, 0]]
    post["cache_lambda"][0:3] = [[10, 0, 0, 0], [20, 0, 0, 0], [30, 0, 0, 0]]
    post["cache_key"][C] = [0, 3, 7]
    post["cache_p"][C] = [0.6, 0, 0]  # moved 0.1 m: no match
    post["cache_lambda"][C] = [40, 0, 0, 0]
    m = bench.merged_cache(S, post, C, 0.01)
    assert list(m["cache_count"]) == [3, 1]
    assert np.array_equal(m["cache_key"], post["cache_key"])
    assert list(m["cache_lambda"][0:3, 0]) == [1, 20, 2]
    assert m["cache_lambda"][C, 0] == 40
    assert np.allclose(m["cache_p"][C], [0.6, 0, 0])


def test_tune_summary_sorts_the_last_phase_by_option():
    """The tuner's last phase (whole-step times only: the stage times read 0) reported
    per partition count, for the ABA kernels in sequence and for the fused step kernel;
    each kernel's tuned and default-shape times from the earlier phases."""
    base = {f: 0 for fs in bench.KERNEL_FIELDS.values() for f in fs}
    base.update(partitions=1, aba_overlap=1, fused=0)

    def trial(ms, **kw):
        return {"shape": dict(base, **kw), "ms": ms}

    rep = {"steps_taken": 15, "chosen_ms": {"collide": 0.05, "rows": 0.03, "pgs": 0.13, "aba": 0.04, "step": 0.21},
           "trials": [trial([0.05, 0.03, 0.14, 0.25, 0.04]), trial([0.06, 0.04, 0.13, 0.26, 0.05], pgs_warps=8),
                      trial([0.0, 0.0, 0.0, 0.21, 0.0]), trial([0.0, 0.0, 0.0, 0.23, 0.0], partitions=2),
                      trial([0.0, 0.0, 0.0, 0.24, 0.0], partitions=4), trial([0.0, 0.0, 0.0, 0.22, 0.0], aba_overlap=0),
                      trial([0.0, 0.0, 0.0, 1.06, 0.0], fused=1)]}
    out = bench.tune_summary(dict(base), rep)
    assert out["partitions_ms"] == {"1": 0.21, "2": 0.23, "4": 0.24}
    assert out["aba_in_sequence_ms"] == 0.22 and out["fused_ms"] == 1.06
    assert out["kernels"]["pgs"] == {"tuned_ms": 0.13, "default_ms": pytest.approx(0.14)}
    assert out["steps_taken"] == 15 and out["trials"] == 7 and out["step_tuned_ms"] == 0.21
