"""Launch shapes and the autotuner (batching of uneven environments).

Every environment runs the same code on one warp (or, in PGS, on one lane
group of 16 or 8 lanes) whatever the shape, so a step must give bit-identical
results under every launch shape: warps per block, plain or persistent grid
(work queue, optionally with SMs reserved for the heaviest environments), LPT
order on or off, lanes per environment, register build, shared-memory staging
capacities (small ones send most rows through the global-memory paths), and the
split of the batch into partitions whose kernels run on parallel graph branches
(each partition's environments see offset views of the per-environment arrays),
the ABA kernels on a side stream beside forward kinematics and collision, and the
fused step kernel that carries each environment through every stage of all the
steps of a call in one launch.
The autotuner's steps are real physics steps and must advance the batch exactly
as plain steps do.
"""
import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(collide_warps=1, collide_persistent=1, rows_warps=1, rows_persistent=1, pgs_warps=1, pgs_persistent=1,
         pgs_lpt=0, pgs_lanes=8, pgs_min_blocks=2, pgs_heavy_sms=0, pgs_stage_contacts=0, pgs_stage_pool=0, aba_lanes=32, partitions=1, aba_overlap=1, fused=0),
    dict(collide_warps=8, collide_persistent=1, rows_warps=8, rows_persistent=1, pgs_warps=2, pgs_persistent=1,
         pgs_lpt=1, pgs_lanes=16, pgs_min_blocks=2, pgs_heavy_sms=0, pgs_stage_contacts=0, pgs_stage_pool=0, aba_lanes=32,
         partitions=3, aba_overlap=0, fused=0),
    dict(collide_warps=2, collide_persistent=0, rows_warps=2, rows_persistent=0, pgs_warps=2, pgs_persistent=0,
         pgs_lpt=0, pgs_lanes=32, pgs_min_blocks=3, pgs_heavy_sms=0, pgs_stage_contacts=8, pgs_stage_pool=1, aba_lanes=16,
         partitions=2, aba_overlap=1, fused=0),
    dict(collide_warps=4, collide_persistent=0, rows_warps=4, rows_persistent=0, pgs_warps=1, pgs_persistent=0,
         pgs_lpt=1, pgs_lanes=16, pgs_min_blocks=2, pgs_heavy_sms=0, pgs_stage_contacts=0, pgs_stage_pool=0, aba_lanes=16,
         partitions=1, aba_overlap=0, fused=0),
    dict(collide_warps=4, collide_persistent=1, rows_warps=4, rows_persistent=1, pgs_warps=4, pgs_persistent=1,
         pgs_lpt=1, pgs_lanes=32, pgs_min_blocks=2, pgs_heavy_sms=19, pgs_stage_contacts=0, pgs_stage_pool=0, aba_lanes=32,
         partitions=4, aba_overlap=1, fused=0),
    dict(collide_warps=2, collide_persistent=1, rows_warps=2, rows_persistent=1, pgs_warps=1, pgs_persistent=1,
         pgs_lpt=1, pgs_lanes=32, pgs_min_blocks=1, pgs_heavy_sms=9, pgs_stage_contacts=72, pgs_stage_pool=64, aba_lanes=32,
         partitions=2, aba_overlap=0, fused=0),
    # the whole step as one persistent launch: LPT order with default staging; environment
    # order with staging small enough that most rows take the global-memory paths
    dict(collide_warps=4, collide_persistent=0, rows_warps=4, rows_persistent=0, pgs_warps=4, pgs_persistent=0,
         pgs_lpt=1, pgs_lanes=32, pgs_min_blocks=2, pgs_heavy_sms=0, pgs_stage_contacts=0, pgs_stage_pool=0, aba_lanes=32,
         partitions=1, aba_overlap=1, fused=1),
    dict(collide_warps=4, collide_persistent=0, rows_warps=4, rows_persistent=0, pgs_warps=4, pgs_persistent=0,
         pgs_lpt=0, pgs_lanes=32, pgs_min_blocks=2, pgs_heavy_sms=0, pgs_stage_contacts=8, pgs_stage_pool=1, aba_lanes=32,
         partitions=1, aba_overlap=0, fused=1),
]


def _sim(batch, params, **kw):
    from paper_2106_14405_gb300 import Sim
    return Sim(batch, params, **kw)


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def _stats_equal(s1, s2):
    a, b = s1.stats(), s2.stats()
    for k in ("n_contacts", "n_rows", "iters", "status"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("use_graph", [False, True])
def test_results_do_not_depend_on_launch_shape(use_graph):
    # uneven scenes (2-40 objects, 0-6 receptacles); enough environments that the
    # persistent grids hand several environments to each warp
    b = sg.make_batch(3, 4096)
    p = sg.params_for(3)
    ref = _sim(b, p, use_graph=use_graph)
    ref.step(12)
    want = ref.get_state()
    for shape in SHAPES:
        s = _sim(b, p, use_graph=use_graph)
        s.set_launch_shape(**shape)
        assert s.launch_shape() == shape
        s.step(5)
        s.step(7)
        _same(want, s.get_state())
        _stats_equal(ref, s)


def test_persistent_queue_resets_between_launches():
    """Persistent launches of different shapes in a row (each must find its
    queue counters at zero) still reproduce the default schedule."""
    b = sg.make_batch(2, 2048)
    p = sg.params_for(2)
    ref = _sim(b, p)
    s = _sim(b, p)
    for i in range(6):
        s.set_launch_shape(**SHAPES[(0, 4, 2)[i % 3]])
        s.step(1)
        ref.step(1)
        _same(ref.get_state(), s.get_state())


def test_autotune_steps_are_plain_steps():
    b = sg.make_batch(3, 1024)
    p = sg.params_for(3)
    s = _sim(b, p, use_graph=True)
    rep = s.autotune(steps_per_trial=1, rounds=2)
    n = rep["steps_taken"]
    # each round's trials run from the same saved state, the batch advancing by the last
    # trial's steps: phases 1-3 (rounds + 1) steps each, phase 4 (whole-step times only)
    # twice that
    n4 = sum(1 for t in rep["trials"] if t["ms"][0] == t["ms"][1] == t["ms"][2] == 0.0)
    p4 = rep["trials"][-n4:]
    assert n4 == 5 and [(t["shape"]["partitions"], t["shape"]["aba_overlap"], t["shape"]["fused"]) for t in p4] == [
        (1, 1, 0), (2, 1, 0), (4, 1, 0), (1, 0, 0), (1, 1, 1)]
    assert n == 3 * 3 + 2 * 3 and len(rep["trials"]) >= 8
    assert all(v > 0 for v in rep["chosen_ms"].values())
    chosen = rep["chosen"]
    assert s.launch_shape() == chosen
    assert chosen["pgs_warps"] in (1, 2, 4, 8) and chosen["pgs_lpt"] in (0, 1) and chosen["pgs_lanes"] in (8, 16, 32)
    ref = _sim(b, p)
    ref.step(n)
    _same(ref.get_state(), s.get_state())
    # the tuned shape runs in the captured graph and keeps matching
    s.step(4)
    ref.step(4)
    _same(ref.get_state(), s.get_state())


def test_invalid_launch_shape_is_rejected():
    from paper_2106_14405_gb300 import SimError
    s = _sim(sg.make_batch(2, 16), sg.params_for(2))
    before = s.launch_shape()
    for bad in (dict(pgs_warps=3), dict(collide_warps=16), dict(rows_persistent=2), dict(pgs_lpt=-1),
                dict(pgs_lanes=4), dict(pgs_lanes=16, pgs_min_blocks=3), dict(pgs_min_blocks=4),
                dict(pgs_lanes=16, pgs_min_blocks=1), dict(pgs_min_blocks=0),
                dict(pgs_heavy_sms=8, pgs_persistent=0), dict(pgs_heavy_sms=-1), dict(pgs_stage_contacts=-1),
                dict(pgs_stage_contacts=256, pgs_stage_pool=64, pgs_warps=8), dict(aba_lanes=8),
                dict(partitions=0), dict(partitions=5), dict(aba_overlap=2), dict(aba_overlap=-1), dict(fused=2),
                dict(fused=1, partitions=2)):
        with pytest.raises(SimError):
            s.set_launch_shape(**bad)
        assert s.launch_shape() == before
    with pytest.raises(SimError):
        s.autotune(steps_per_trial=0)
    two = _sim(sg.make_batch(2, 2), sg.params_for(2))
    with pytest.raises(SimError):
        two.set_launch_shape(partitions=3)  # more partitions than environments


def test_partitions_with_the_learned_warm_start_and_residual_mode():
    """Partitions on parallel graph branches with the learned warm start (each
    partition lists its own network rows) and a residual target: bit-identical to
    the unpartitioned step, statistics included."""
    b = sg.make_batch(2, 1024)
    p = sg.params_for(4)
    p.warm_mode = 2
    P = sg.mlp_init(2) * 0.1
    out = []
    for parts in (1, 2, 4):
        s = _sim(b, p, use_graph=True)
        s.set_mlp(P)
        s.set_launch_shape(partitions=parts, pgs_persistent=1, pgs_heavy_sms=8)
        s.step(6)
        s.step(3)
        out.append((s.get_state(), s.stats()))
    for st, stats in out[1:]:
        _same(out[0][0], st)
        for k in ("n_contacts", "n_rows", "iters", "status", "n_colours"):
            assert np.array_equal(out[0][1][k], stats[k]), k


def test_fused_step_matches_the_stage_kernels():
    """The fused step kernel against the stage kernels on the mobile-manipulator
    workload (9-joint arms, receptacles): bit-identical state and statistics after
    calls of different step counts, with and without graph capture, over enough
    steps for the arms to press into clutter; warm mode 2 under a fused shape runs the
    stage kernels (the same results again)."""
    b = sg.make_batch(2, 2048)
    p = sg.params_for(2)
    for use_graph in (False, True):
        ref = _sim(b, p, use_graph=use_graph)
        s = _sim(b, p, use_graph=use_graph)
        s.set_launch_shape(fused=1, pgs_stage_contacts=16, pgs_stage_pool=8)
        for n in (1, 6, 3, 30):
            ref.step(n)
            s.step(n)
            _same(ref.get_state(), s.get_state())
            _stats_equal(ref, s)
    p2 = sg.params_for(2)
    p2.warm_mode = 2
    P = sg.mlp_init(2) * 0.1
    out = []
    for fused in (0, 1):
        s = _sim(b, p2, use_graph=True)
        s.set_mlp(P)
        s.set_launch_shape(fused=fused)
        s.step(4)
        out.append(s.get_state())
    _same(out[0], out[1])


def test_profiling_modes():
    """Mode 1 times every stage; mode 2 only the PGS kernel (the other stages read
    0 ms); both leave the results unchanged; other modes are refused."""
    from paper_2106_14405_gb300 import SimError
    b = sg.make_batch(2, 256)
    p = sg.params_for(2)
    ref = _sim(b, p, use_graph=True)
    ref.step(8)
    for mode in (True, "pgs"):
        s = _sim(b, p, use_graph=True)
        s.set_profiling(mode)
        s.step(4)
        ms, ln = s.kernel_times()
        s.step(4)
        assert ms["pgs"] > 0 and ln["pgs"] == 4
        if mode == "pgs":
            assert all(ms[k] == 0.0 for k in ms if k != "pgs")
        else:
            assert ms["aba"] > 0 and ms["collide"] > 0 and ms["rows"] > 0
        _same(ref.get_state(), s.get_state())
        with pytest.raises(SimError):
            s.set_profiling(3)
