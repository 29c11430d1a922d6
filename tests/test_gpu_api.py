"""Boundary calls beyond the step itself, through the C ABI on the GPU: the batch
totals (sim_get_stats) against the per-environment statistics, the warm-start
setter (sim_set_warm_start) against the equivalent parameter path, the training
log's row rules (only converged solves), the trainer's data preparation against
NumPy, the library's FP32 throughput probe, and each handle keeping its device."""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


def _sim(b, p, **kw):
    from paper_2106_14405_gb300 import Sim
    return Sim(b, p, **kw)


def test_batch_totals_equal_the_sums_of_the_per_env_statistics():
    b = sg.make_batch(3, 512)  # doors and drawers: contacts on articulation links
    p = sg.params_for(3)
    p.pgs_tol, p.pgs_max_iters = 1e-6, 1000  # residual mode: sweep counts vary per environment
    sim = _sim(b, p)
    sim.step(40)
    t = sim.totals()
    st = sim.stats()
    s = sim.get_state()
    assert t["n_envs"] == 512
    assert t["sum_iters"] == int(st["iters"].astype(np.int64).sum())
    assert t["max_iters"] == int(st["iters"].max())
    assert t["row_sweeps"] == int((st["iters"].astype(np.int64) * st["n_rows"]).sum())
    assert t["n_contacts"] == int(st["n_contacts"].sum())
    assert t["n_rows"] == int(st["n_rows"].sum())
    assert t["n_limit_rows"] == int(st["n_limit_rows"].sum())
    assert t["n_iter_cap"] == int(((st["status"] & 4) != 0).sum())
    assert t["n_fp64"] == int((st["fp64_used"] != 0).sum())
    assert t["max_colours"] == int(st["n_colours"].max())
    assert t["status_or"] == int(np.bitwise_or.reduce(st["status"].astype(np.int64)))
    assert t["n_awake"] == int(s["obj_awake"].sum())
    assert t["max_resid"] == pytest.approx(float(st["resid"].max()), rel=0, abs=0)
    # articulation row endpoints: one per contact endpoint on an articulation link (at
    # most 64 per environment)
    c = sim.contact_keys()
    nobj = np.diff(b["obj_off"])
    jo = b["joint_off"][b["art_off"]]
    nlink = np.diff(jo)
    slots = 0
    for e in range(b.n_envs):
        k = c["key"][e, :c["count"][e]]
        link = lambda x: (x >= nobj[e]) & (x < nobj[e] + nlink[e])
        slots += min(64, int(link(k[:, 0]).sum() + link(k[:, 1]).sum()))
    assert t["n_pool_slots"] == slots and slots > 0


def test_set_warm_start_equals_the_parameter_path():
    """sim_set_warm_start(cold / prior / learned with a network) steps bit-identically
    to a handle created with that warm_mode (and sim_set_mlp); learned without a
    network is refused with SIM_ERR_STATE."""
    from paper_2106_14405_gb300._native import SimError
    b = sg.make_batch(2, 64)
    P = sg.mlp_init(3) * 0.2
    base = _sim(b, sg.params_for(2))
    base.step(20)
    s0 = base.get_state()
    for mode, name in ((0, "cold"), (2, "learned"), (1, "prior")):
        q = sg.params_for(2)
        q.warm_mode = mode
        ref = _sim(b, q)
        if mode == 2:
            ref.set_mlp(P)
        ref.set_state(s0)
        ref.step(3)
        sim = _sim(b, sg.params_for(2))
        if mode == 2:
            with pytest.raises(SimError, match="SIM_ERR_STATE"):
                sim.set_warm_start("learned")
        sim.set_warm_start(name, P if mode == 2 else None)
        sim.set_state(s0)
        sim.step(3)
        a, r = sim.get_state(), ref.get_state()
        for k in ("obj_pos", "obj_vel", "obj_omega", "joint_qd", "cache_lambda"):
            assert np.array_equal(a[k], r[k]), (name, k)


def test_log_keeps_only_converged_solves():
    """In residual mode the training log holds the contacts of the environments whose
    solve met the residual target, and no others."""
    b = sg.make_batch(2, 256)
    p = sg.params_for(4)
    p.pgs_max_iters = 12  # many solves stop at the cap
    sim = _sim(b, p, log_features=True)
    sim.step(30)
    f, l, n = sim.log_contacts(1 << 16)
    st = sim.stats()
    conv = st["resid"] <= p.pgs_tol
    assert 0 < conv.sum() < len(conv)
    assert n == int(st["n_contacts"][conv].sum())
    assert torch.isfinite(l).all() and torch.isfinite(f).all()


def test_training_rows_and_feature_statistics_match_numpy():
    """mlp_select_rows keeps the rows with finite targets (and, when asked, only those
    the warm start serves: feature 26 = 0 or |features 9-11| > gate), in order, targets
    clipped; mlp_feature_stats gives the per-feature mean and standard deviation."""
    from paper_2106_14405_gb300.learn import feature_stats, select_rows
    rng = np.random.default_rng(11)
    n = 100_003
    X = rng.normal(size=(n, 32)).astype(np.float32)
    X[:, 26] = rng.random(n) < 0.7
    X[:, 5] = 3.5  # a constant feature: its deviation is reported as 1
    T = (rng.normal(size=(n, 3)) * 8).astype(np.float32)
    T[rng.random(n) < 0.01, 1] = np.nan
    T[rng.random(n) < 0.01, 2] = np.inf
    gate = 1.3
    for only_used in (False, True):
        keep = np.isfinite(T).all(1)
        if only_used:
            keep &= (X[:, 26] == 0) | (np.sqrt((X[:, 9:12].astype(np.float32) ** 2).sum(1)) > gate)
        Xo, To = select_rows(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), only_used, gate, 10.0)
        assert Xo.shape[0] == keep.sum()
        assert np.array_equal(Xo.cpu().numpy(), X[keep])
        assert np.array_equal(To.cpu().numpy(), np.clip(T[keep], -10, 10))
    mean, std = feature_stats(torch.from_numpy(X).cuda())
    ref_std = X.astype(np.float64).std(0)
    ref_std[ref_std < 1e-6] = 1.0
    np.testing.assert_allclose(mean, X.astype(np.float64).mean(0), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(std, ref_std, rtol=1e-6)
    assert std[5] == 1.0


def test_fp32_fma_peak_is_plausible():
    """The library's own FP32 throughput probe: between a quarter and 1.2 times the
    nominal peak (SMs x 128 FP32 lanes x 2 flops x the maximum SM clock)."""
    from paper_2106_14405_gb300.engine import fp32_fma_peak
    tf, ms = fp32_fma_peak(iters=1024, reps=3)
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.1e9 / 1e12
    assert 0.25 * nominal < tf < 1.2 * nominal, (tf, nominal)
    assert ms > 0


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs two GPUs")
def test_handle_keeps_its_device():
    """A handle created on device 1 works while device 0 is current, and every call
    leaves the caller's current device as it was."""
    b = sg.make_batch(2, 16)
    torch.cuda.set_device(1)
    with torch.cuda.device(1):
        sim = _sim(b, sg.params_for(2))
    torch.cuda.set_device(0)
    sim.step(2)
    rc, _, _ = sim.sync()
    assert rc == 0 and torch.cuda.current_device() == 0
    s = sim.get_state()
    assert np.isfinite(s["obj_pos"]).all() and torch.cuda.current_device() == 0


def test_last_error_is_kept_per_handle():
    """sim_last_error(h) holds the last error of a call on h; another handle's stays
    empty, and NULL gives the thread's last error."""
    import ctypes
    from paper_2106_14405_gb300 import SimError, _native as N
    lib = N.load()
    a = _sim(sg.make_batch(2, 4), sg.params_for(2))
    b = _sim(sg.make_batch(2, 4), sg.params_for(2))
    with pytest.raises(SimError):
        a.set_launch_shape(pgs_warps=3)
    assert b"pgs_warps" in lib.sim_last_error(a.h)
    assert lib.sim_last_error(b.h) == b""
    assert b"pgs_warps" in lib.sim_last_error(None)
    n = ctypes.c_int(0)
    assert lib.sim_log_contacts_noalloc(b.h, None, None, 4, ctypes.byref(n)) == 7  # no features logged
    assert b"log_features" in lib.sim_last_error(b.h)
    assert b"pgs_warps" in lib.sim_last_error(a.h)
