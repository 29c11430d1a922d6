"""The multi-rank path of bench.py on CPU: two `gloo` ranks.

Environments never interact, so N ranks run N independent batches (weak
scaling): each rank draws its own scenes (seed offset by rank), nothing is
exchanged on the data path, and the job's time is the max over ranks, reduced
once after the timed region.  These tests run that host logic with world size
2 on the gloo backend; the GPU work itself is not involved.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import scenegen as sg

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.rank_layout()
    E = 6
    b = sg.make_batch(2, E, seed_offset=bench.rank_seed_offset(r, E))
    # a rank-specific "timed region": the slowest rank sets the job's time
    my_s = 0.25 + 0.5 * r
    job_s = bench.max_over_ranks(my_s)
    rate = bench.whole_job_rate(w, E, 4 * 3, job_s)
    res = {"layout": [w, r, lr], "job_s": job_s, "rate": rate,
           "obj_pos": b.arrays["obj_pos"].tolist(), "obj_off": b.arrays["obj_off"].tolist()}
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_whole_job_rate_and_distinct_scenes(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["layout"] == [2, 0, 0] and r1["layout"] == [2, 1, 1]
    # both ranks see the max over ranks, and the whole-job rate counts both ranks' environments
    assert r0["job_s"] == r1["job_s"] == 0.75
    assert r0["rate"] == pytest.approx(2 * 6 * 12 / 0.75)
    # same workload structure, different scenes (seeded per rank)
    assert r0["obj_off"] == r1["obj_off"]
    assert not np.allclose(np.array(r0["obj_pos"]), np.array(r1["obj_pos"]))


def test_single_process_reduces_to_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.rank_seed_offset(0, 4096) == 0 and bench.rank_seed_offset(3, 4096) == 3 * 4096
    assert bench.whole_job_rate(1, 4096, 4, 0.002) == pytest.approx(4096 * 4 / 0.002)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle arm is timed by rank 0 alone; another rank exits 0
    without work and prints nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
