#!/usr/bin/env python
"""Throughput of the batched physics step on GB300: env physics steps per second.

Workload (default): 4096 mobile-manipulator environments, each with 10 dropped
objects on 20 static receptacle boxes, PGS at 10 sweeps, dt = 1/120 s,
sleeping on, prior-frame warm start.  One benchmark step = 15 physics steps
(1/8 s of simulated time: 3.75 of the paper's 1/30 s simulation steps of 4 x
1/120 s physics, without rendering) in one sim_step call replayed from a CUDA
graph, so that the default K = 20 steps time the workload's 300 physics steps
after 60.  The 65536-env batch, whose joint targets follow a random walk
refreshed every 4 physics steps, steps 4 physics steps per benchmark step.
Inputs are synthetic (seeded scenes).

Timed window: the scene is advanced 60 physics steps from its initial state,
and that state is saved.  The autotuner (launch shapes) and the W warm-up steps
run from it and the state is restored after each, so the K timed steps are
always physics steps 60 .. 60 + 15 K of the workload (60-360 at the default
K = 20).  The per-stage pass and the end-to-end pass replay the same window.
The uneven 16384-env batch and the 65536-env batch with the learned warm start
are measured the same way and reported as extra keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With torchrun (N > 1) every rank simulates its own
environments (weak scaling, no collective on the data path); rank 0 prints the
line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen as sg  # noqa: E402

METRIC = "env physics steps/s on 1 GB300 (plain vs learned warm-start @1e-6 resid); % roofline"
UNIT = "env-steps/s"
# the paper's simulation step: 4 physics steps of 1/120 s per 1/30 s (Sec. 4.4); workload
# 5 refreshes its joint targets at this period (4 substeps per target refresh)
CONTROL_SUBSTEPS = 4
# physics steps per benchmark step: 15 where the joint targets stay fixed (300 timed
# physics steps at the default K = 20), one target refresh period for workload 5
STEP_PHYSICS = {2: 15, 3: 15, 5: CONTROL_SUBSTEPS}
WINDOW_START = 60  # physics steps before the timed window
ENVS = {2: 4096, 3: 16384, 5: 65536}
# the warm-start network's training scenes: seeds disjoint from every rank's benchmark
# scenes (up to 8 x 65536 envs) and from the held-out scenes of the warm-start study
TRAIN_SEED_OFFSET = 2_000_000
HELD_OUT_OFFSET = 500_000
TRAIN_PAIRS = 10_000_000  # logged contact-impulse pairs the study's network is trained on
LEARN_GATE = 4.0          # matched contacts served by the network: |v_rel| > LEARN_GATE |g| dt
HBM_FALLBACK_GBS = 6800.0
# Algorithmic global-memory bytes of the PGS launch (staging, write-back and the
# integration it carries), per item, from the SoA layout: an object reads its predicted
# velocities, inverse mass / inertia, orientation, position and compensation, awake flag
# and sleep counter (104 B) and writes velocities, position, compensation, orientation
# and counter (84 B); a joint reads its predicted rate, coordinate, compensation and
# articulation index (16 B) and writes rate, coordinate, compensation and limit / motor
# state (24 B); a contact reads its row (normal, tangent, effective masses, lever arms,
# endpoint codes, warm start: 104 B) and, in the write-back, normal, tangent, key and
# point (64 B), and writes its impulses and its cache entry (64 B); an articulation row
# endpoint is one 288 B record (J and M~^-1 J^T rows of 9, padded to 12); a limit row
# reads 68 B and writes 8 B; an environment reads its counts and offsets and writes its
# statistics (40 B).
PGS_BYTES = {"object": 188, "joint": 40, "contact": 232, "pool_slot": 288, "limit_row": 76, "env": 40}
# DRAM bytes (read + write) of one k_pgs launch of the default workload at the tuned
# launch shape, the timed window's first physics step, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), with a digest of the kernel's sources
# at capture time: reported as roofline.traffic only while the sources are unchanged
# (a changed kernel reports null).
PGS_TRAFFIC = {"bytes": 25082880 + 7168, "config": 2, "envs": 4096, "sources_sha256_16": "b1025e03092ec198",
               "sources": ("paper_2106_14405_gb300/csrc/k_solve.cu", "paper_2106_14405_gb300/csrc/solve.cuh",
                           "paper_2106_14405_gb300/csrc/sim_internal.cuh")}
STAGES = ("aba", "collide", "rows", "mlp", "lpt", "pgs", "integrate")
WARM = {"cold": 0, "prior": 1, "learned": 2}


def pgs_traffic(cfg, E):
    """DRAM bytes per PGS launch from the ncu capture, for the workload it was taken on
    and while the kernel's sources are unchanged since; else None."""
    if (cfg, E) != (PGS_TRAFFIC["config"], PGS_TRAFFIC["envs"]):
        return None
    import hashlib
    h = hashlib.sha256()
    for f in PGS_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return PGS_TRAFFIC["bytes"] if h.hexdigest()[:16] == PGS_TRAFFIC["sources_sha256_16"] else None


def pgs_bytes(totals, n_objects, n_joints):
    """Algorithmic bytes of one PGS launch from the step's totals (sim_get_stats)."""
    B = PGS_BYTES
    return (B["object"] * n_objects + B["joint"] * n_joints + B["contact"] * totals["n_contacts"] +
            B["pool_slot"] * totals["n_pool_slots"] + B["limit_row"] * totals["n_limit_rows"] +
            B["env"] * totals["n_envs"])


def step_physics(cfg):
    """Physics steps per benchmark step of workload cfg."""
    return STEP_PHYSICS.get(cfg, 15)


def timed_window(warmup, steps, cfg=2):
    """Physics steps [first, last) of the timed region: the window starts at
    WINDOW_START whatever the warm-up (warm-up and tuning run from the saved start)."""
    return WINDOW_START, WINDOW_START + step_physics(cfg) * steps


BF16_FALLBACK_TFLOPS = 1700.0
# FLOPs of one contact through the network: 2 x (32 x 128 + 128 x 128 + 128 x 128) on the
# tensor cores and 2 x 128 x 3 for the output layer on the CUDA cores
MLP_FLOP_PER_ROW = 2 * (32 * 128 + 128 * 128 + 128 * 128) + 2 * 128 * 3


def bf16_peak():
    """(TFLOP/s, source): the measured sustained cuBLAS BF16 rate of MEASURED_PEAKS.json
    (the inference kernel runs inside a long step), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops_sustained"])
        return v, "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except Exception:
        return BF16_FALLBACK_TFLOPS, "of fallback"


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "of fallback"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--envs", type=int, default=None)
    ap.add_argument("--extra-configs", default="3,5", help="workloads also measured as extra keys ('' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm-start-study", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--shape", default=None, help="launch shape as JSON (fields of SimLaunchShape); skips the autotuner")
    ap.add_argument("--warm-start", default=None, choices=("cold", "prior", "learned"),
                    help="PGS warm start (default: learned for workload 5, which specifies it, else prior-frame); "
                         "learned trains the network first with the library's kernels")
    return ap.parse_args(argv)


def workload_name(cfg, E):
    return {2: f"mobile-manipulator rearrangement, {E} envs x (9-DoF arm + 10 objects + 20 static boxes), "
               f"PGS 10 sweeps, dt 1/120, sleeping, prior-frame warm start",
            3: f"uneven batch, {E} envs x (2..40 objects, 0..6 doors/drawers), PGS 10 sweeps, dt 1/120",
            5: f"large, {E} envs x (30 objects, 4 doors/drawers), dt 1/240, random-walk targets, "
               f"learned warm start"}.get(cfg, f"workload {cfg}, {E} envs")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- ranks
def rank_layout():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed_offset(rank, envs_per_rank):
    """Scene seed offset of a rank: every rank simulates its own environments
    (weak scaling), none shared, no exchange between ranks on the data path."""
    return rank * envs_per_rank


def max_over_ranks(x, device=None):
    """Max of x over the ranks of the default process group (x itself when there
    is none or it has one rank): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, envs_per_rank, physics_steps, seconds):
    """Env physics steps per second of the whole job: all ranks' environments over
    the max-over-ranks time."""
    return world * envs_per_rank * physics_steps / seconds


def default_warm_start(cfg):
    """Workload 5 specifies the learned warm start; the others run the prior-frame one."""
    return "learned" if cfg == 5 else "prior"


# ----------------------------------------------------------------------------- the oracle (CPU legs only)
def oracle_for(cfg, E, warm, mlp=None, batch=None, **kw):
    """The FP64 oracle on E envs of workload `cfg` (or on `batch`) with the given warm
    start; in learned mode with the network `mlp` (a seeded one when None: at a fixed
    sweep count the work per step does not depend on the weights)."""
    import oracle as O
    b = batch if batch is not None else sg.make_batch(cfg, E)
    p = sg.params_for(cfg)
    p.warm_mode = WARM[warm]
    o = O.Oracle(b, p, **kw)
    if warm == "learned":
        o.set_mlp(sg.mlp_init(0) if mlp is None else mlp)
    return o


def oracle_run(cfg, E, warm_steps, timed_steps, threads, warm="prior", min_s=10.0, max_s=30.0, start=None,
               batch=None, mlp=None):
    """Time the FP64 oracle on the host cores over E envs: `timed_steps` physics steps,
    repeated (from the same start state when given, else continuing) until about `min_s`
    seconds of work and not past about `max_s`; returns (env-steps/s, seconds, steps)."""
    o = oracle_for(cfg, E, warm, mlp=mlp, batch=batch)
    if start is not None:
        o.set_state(start)
    else:
        o.step(warm_steps, threads)
    chunk = max(1, timed_steps)
    done, dt = 0, 0.0
    while done == 0 or (dt < min_s and dt * (done + chunk) / done <= max_s):
        if start is not None and done:
            o.set_state(start)
        t0 = time.perf_counter()
        o.step(chunk, threads)
        dt += time.perf_counter() - t0
        done += chunk
    return o.E * done / dt, dt, done


def oracle_op_counts(cfg, E, warm_steps, timed_steps, warm="prior", start=None, batch=None, mlp=None, threads=1):
    """Algorithmic FP operations per env-step per stage, counted by the op-counting
    oracle build over `timed_steps` physics steps (from `start` when given), with the
    oracle's PGS row updates (rows x sweeps) per env-step."""
    o = oracle_for(cfg, E, warm, mlp=mlp, batch=batch, counting=True)
    if start is not None:
        o.set_state(start)
    else:
        o.step(warm_steps, threads)
    o.reset_op_counts()
    row_sweeps = 0
    for _ in range(timed_steps):
        o.step(1, threads)
        st = o.stats()
        row_sweeps += int((st["n_rows"].astype(np.int64) * st["iters"]).sum())
    c = o.op_counts()
    out = {k: v / (o.E * timed_steps) for k, v in c.items()}
    out["row_sweeps"] = row_sweeps / (o.E * timed_steps)
    return out


def oracle_start(gs):
    """The oracle state from an engine state (positions read as value - compensation)."""
    from oracle.compare import compensated, gpu_to_oracle
    return gpu_to_oracle(compensated(gs))


def cpu_leg(wl, K, threads, full):
    """The benchmark's CPU leg for one workload: the oracle timed over the timed window
    (`full`: all environments, repeated from the window's start for 10-30 s), the
    op-counting oracle over the window's environments and steps (a sample of 1024
    environments over the whole window for the large workloads), and the per-output
    errors of one engine step from the window's end against the oracle."""
    from oracle.compare import sampled_parity, subset_state
    out = {}
    start = oracle_start(wl.S0_host)
    steps = wl.sub * K
    if full:
        rate, secs, done = oracle_run(wl.cfg, wl.E, 0, steps, threads, wl.warm, start=start, batch=wl.b, mlp=wl.mlp)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"{wl.E} envs of the same workload from the timed window's first state "
                                         f"(physics step {WINDOW_START}), the window's {steps} physics steps "
                                         f"repeated: {done} steps, {threads} host threads, {secs:.2f} s"}
    if full:
        cnt_envs, cnt_steps, cb, cs = np.arange(wl.E), steps, wl.b, start
    else:
        rng = np.random.default_rng(7)
        cnt_envs = np.sort(rng.choice(wl.E, min(wl.E, 1024), replace=False))
        cnt_steps = steps
        cb, cs = wl.b.subset(cnt_envs), subset_state(wl.b, wl.S0_host, cnt_envs)
    t0 = time.perf_counter()
    out["counts"] = oracle_op_counts(wl.cfg, len(cnt_envs), 0, cnt_steps, wl.warm, start=cs, batch=cb, mlp=wl.mlp,
                                     threads=threads)
    out["count_sample"] = (f"{len(cnt_envs)} envs x {cnt_steps} physics steps from the timed window's first "
                           f"state, op-counting oracle ({time.perf_counter() - t0:.1f} s)")
    # per-output errors: one step from the window's end state, sampled envs + the heaviest
    rng = np.random.default_rng(0)
    envs = np.unique(np.concatenate([rng.choice(wl.E, min(wl.E, 64), replace=False), [wl.heaviest]]))
    p = sg.params_for(wl.cfg)
    p.warm_mode = WARM[wl.warm]
    if wl.warm == "learned":  # BF16 predictions: compare where the solution no longer depends on the start
        p.pgs_tol, p.pgs_max_iters = 1e-6, 1000
    par = sampled_parity(wl.b, p, wl.P_start, wl.P_after, wl.P_contacts, envs, mlp=wl.mlp)
    par["step"] = (f"one physics step from the state at the end of the timed window (Kahan compensations "
                   f"cleared), {len(envs)} envs: 64 sampled and the one with the longest colour x sweep chain"
                   + ("; both engines iterate to the 1e-6 residual (BF16 network)" if wl.warm == "learned" else ""))
    out["parity"] = par
    return out


# ----------------------------------------------------------------------------- warm-start network
def train_warm_start_network(cfg=2, pairs=TRAIN_PAIRS, envs=8192, epochs=8):
    """The learned warm start's network, trained by the library's own kernels on the
    impulses the plain solver logs when iterated to the 1e-6 residual (only converged
    solves are logged), on scenes of workload `cfg` (2: the mobile-manipulator
    workload) drawn from seeds disjoint from the benchmark's, until `pairs` contact
    pairs are logged; returns (params, pairs, losses, collect s, train s)."""
    import torch
    from paper_2106_14405_gb300 import Sim
    from paper_2106_14405_gb300.learn import train
    p = sg.params_for(4) if cfg == 2 else sg.params_for(cfg)
    p.pgs_tol, p.pgs_max_iters = 1e-6, 1000
    p.warm_mode = 1
    t0 = time.perf_counter()
    sim = Sim(sg.make_batch(cfg, envs, seed_offset=TRAIN_SEED_OFFSET), p, log_features=True)
    sim.step(20)
    feats, lams, n = [], [], 0
    while n < pairs:
        sim.step(1)
        f, l, _ = sim.log_contacts(1 << 22)
        feats.append(f.clone())
        lams.append(l.clone())
        n += f.shape[0]
        sim.sync()
    sim.close()
    X, T = torch.cat(feats), torch.cat(lams)
    del feats, lams
    t1 = time.perf_counter()
    params, losses = train(X, T, sg.mlp_init(0), epochs=epochs, batch=4096, lr=1e-3)
    t2 = time.perf_counter()
    return params, int(X.shape[0]), losses, t1 - t0, t2 - t1


def merged_cache(S, post, C, match_dist):
    """A warm-start cache holding, for each contact of the step that led from S to post,
    the prior-frame entry where the contact matched one (the prior-frame start) and the
    step's converged impulse where it did not: the start an ideal predictor of the new
    contacts would give."""
    E = len(post["cache_count"])

    def flat(st):
        cnt = np.asarray(st["cache_count"])
        mask = np.arange(C)[None, :] < cnt[:, None]
        key = np.asarray(st["cache_key"]).reshape(E, C, 3)[mask].astype(np.int64)
        env = np.repeat(np.arange(E, dtype=np.int64), cnt)
        code = ((env * 128 + key[:, 0]) * 128 + key[:, 1]) * 4096 + key[:, 2]
        return mask, code

    mS, cS = flat(S)
    mP, cP = flat(post)
    pS = np.asarray(S["cache_p"]).reshape(E, C, 3)[mS]
    lS = np.asarray(S["cache_lambda"]).reshape(E, C, 4)[mS]
    pP = np.asarray(post["cache_p"]).reshape(E, C, 3)[mP]
    lP = np.asarray(post["cache_lambda"]).reshape(E, C, 4)[mP]
    out = {k: np.array(S[k], copy=True) for k in ("cache_count", "cache_key", "cache_p", "cache_lambda")}
    out["cache_count"] = np.array(post["cache_count"], copy=True)
    out["cache_key"] = np.array(post["cache_key"], copy=True)
    lam = lP.copy()
    if len(cS) and len(cP):
        order = np.argsort(cS, kind="stable")
        idx = np.clip(np.searchsorted(cS[order], cP), 0, len(cS) - 1)
        cand = order[idx]
        hit = (cS[cand] == cP) & (np.linalg.norm(pS[cand] - pP, axis=1) < match_dist)
        lam[hit] = lS[cand[hit]]
    cp = out["cache_p"].reshape(E, C, 3)
    cp[mP] = pP
    cl = out["cache_lambda"].reshape(E, C, 4)
    cl[mP] = lam
    return out


def frictionless(batch):
    """The same scenes with every friction coefficient 0."""
    b = sg.Batch(batch.n_envs, {k: np.array(v, copy=True) for k, v in batch.arrays.items()})
    for k in ("obj_mu", "stat_mu", "joint_mu"):
        b.arrays[k][:] = 0.0
    return b


def warm_start_study(eval_envs=4096, eval_steps=8, epochs=20, pairs=TRAIN_PAIRS):
    """Cold / prior-frame / learned warm start iterated to the 1e-6 relative residual
    (cap 1000 sweeps) on held-out scenes of the mobile-manipulator workload, with the
    bounds that explain the result: the sweeps an ideal predictor of the new contacts
    would leave, how many capped solves cap again from their own end state (limit
    cycles of the iteration, which no start removes), and how many converge once
    friction is removed."""
    import torch
    from paper_2106_14405_gb300 import Sim
    p = sg.params_for(4)
    params, n_samples, losses, collect_s, train_s = train_warm_start_network(2, pairs, epochs=epochs)
    held = sg.make_batch(4, eval_envs, seed_offset=HELD_OUT_OFFSET)
    out = {"workload": f"{eval_envs} held-out envs of the mobile-manipulator workload, PGS to 1e-6 relative "
                       f"residual (cap {p.pgs_max_iters} sweeps), {eval_steps} physics steps after 30",
           "train_samples": n_samples, "train_epochs": epochs, "train_loss_per_epoch": losses,
           "collect_s": collect_s, "train_s": train_s, "modes": {}}
    base = Sim(held, p)
    base.step(30)
    start = base.get_state()
    base.close()
    per_mode = {}
    for name in ("cold", "prior", "learned"):
        q = sg.params_for(4)
        q.warm_mode = WARM[name]
        sim = Sim(held, q)
        if name == "learned":
            sim.set_mlp(params)
        sim.set_state(start)
        iters, capped, chain, ms = [], [], [], 0.0
        stream = torch.cuda.current_stream()
        for _ in range(eval_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            st = sim.stats()
            iters.append(np.where(st["n_rows"] > 0, st["iters"], -1))
            capped.append((st["status"] & 4) != 0)
            chain.append(int((st["iters"].astype(np.int64) * np.maximum(st["n_colours"], 1)).max()))
            sim.sync()
        per_mode[name] = (np.stack(iters), np.stack(capped), ms, chain)
        sim.close()
    ok = np.ones_like(per_mode["cold"][0], bool)
    for it, cap, _, _ in per_mode.values():
        ok &= (it >= 0) & ~cap
    for name, (it, cap, ms, chain) in per_mode.items():
        act = it >= 0
        out["modes"][name] = {"mean_sweeps_converged": float(it[ok].mean()),
                              "median_sweeps_converged": float(np.median(it[ok])),
                              "p95_sweeps_converged": float(np.percentile(it[ok], 95)),
                              "mean_sweeps_all": float(it[act].mean()),
                              "cap_hit_frac": float(cap[act].mean()),
                              "env_steps_per_s": eval_envs * eval_steps / (ms / 1e3),
                              "longest_chain_mean": float(np.mean(chain))}
    out["converged_samples"] = int(ok.sum())
    pr, le = out["modes"]["prior"], out["modes"]["learned"]
    out["learned_vs_prior"] = {"sweeps_ratio": le["mean_sweeps_converged"] / pr["mean_sweeps_converged"],
                               "throughput_ratio": le["env_steps_per_s"] / pr["env_steps_per_s"]}
    out["bounds"] = warm_start_bounds(held, start, eval_steps)
    return out


def warm_start_bounds(held, start, eval_steps):
    """Along the prior-frame trajectory from `start`, per step: the same step from an
    ideal start for the new contacts (their converged impulses) and from the step's own
    end state (every impulse at its final value: the start no predictor can beat), and
    the frictionless scene's step; each step's device time with CUDA events."""
    import torch
    from paper_2106_14405_gb300 import Sim
    p = sg.params_for(4)
    sim = Sim(held, p)
    pf = sg.params_for(4)
    pf.plane_mu = 0.0
    fsim = Sim(frictionless(held), pf)
    sim.set_state(start)
    C = int(p.max_contacts)
    keys = ("cache_count", "cache_key", "cache_p", "cache_lambda", "joint_lim_lambda", "joint_lim_side")
    rec = {k: [] for k in ("prior", "ideal_new", "own_end", "frictionless")}
    ms = {k: 0.0 for k in rec}
    stream = torch.cuda.current_stream()

    def timed_step(name):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[name] += e0.elapsed_time(e1)
        rec[name].append(sim.stats())
        sim.sync()

    for _ in range(eval_steps):
        S = sim.get_state()
        timed_step("prior")
        post = sim.get_state()
        sim.set_state({**S, **merged_cache(S, post, C, p.match_dist)})
        timed_step("ideal_new")
        sim.set_state({**S, **{k: post[k] for k in keys}})
        timed_step("own_end")
        fsim.set_state(S)
        fsim.step(1)
        rec["frictionless"].append(fsim.stats())
        fsim.sync()
        sim.set_state(post)
    sim.close()
    fsim.close()

    def arr(name, k):
        return np.stack([s[k] for s in rec[name]])

    act = arr("prior", "n_rows") > 0
    cap = {n: (arr(n, "status") & 4) != 0 for n in rec}
    it = {n: arr(n, "iters") for n in rec}
    both = act & ~cap["prior"] & ~cap["ideal_new"]
    capped = act & cap["prior"]
    rate = {n: held.n_envs * eval_steps / (ms[n] / 1e3) for n in ("prior", "ideal_new", "own_end")}
    conv = act & ~cap["prior"] & ~cap["own_end"]
    return {"prior_env_steps_per_s": rate["prior"],
            "ideal_new_contacts": {"mean_sweeps": float(it["ideal_new"][both].mean()),
                                   "prior_mean_sweeps": float(it["prior"][both].mean()),
                                   "cap_hit_frac": float(cap["ideal_new"][act].mean()),
                                   "env_steps_per_s": rate["ideal_new"],
                                   "note": "new contacts started at their converged impulses, matched ones at the "
                                           "prior frame: the best any predictor of the new contacts can do"},
            "ideal_all_contacts": {"mean_sweeps": float(it["own_end"][conv].mean()),
                                   "prior_mean_sweeps": float(it["prior"][conv].mean()),
                                   "cap_hit_frac": float(cap["own_end"][act].mean()),
                                   "env_steps_per_s": rate["own_end"],
                                   "note": "every impulse started at the step's own converged (or capped) value: "
                                           "the best any warm start can do; the capped limit cycles still set "
                                           "the kernel's length"},
            "capped_env_steps": int(capped.sum()), "prior_cap_hit_frac": float(cap["prior"][act].mean()),
            "capped_again_from_own_end_state": float(cap["own_end"][capped].mean()) if capped.any() else None,
            "capped_converging_without_friction": float((~cap["frictionless"][capped]).mean())
            if capped.any() else None}


# ----------------------------------------------------------------------------- our arm
KERNEL_FIELDS = {"collide": ("collide_warps", "collide_persistent"), "rows": ("rows_warps", "rows_persistent"),
                 "aba": ("aba_lanes",),
                 "pgs": ("pgs_warps", "pgs_persistent", "pgs_lpt", "pgs_lanes", "pgs_min_blocks",
                         "pgs_heavy_sms", "pgs_stage_contacts", "pgs_stage_pool")}


def tune_summary(default, rep):
    """Whole-step ms per physics step at the chosen shape and, per kernel, its tuned and
    default-shape median ms per physics step."""
    out = {"steps_taken": rep["steps_taken"], "trials": len(rep["trials"]), "kernels": {}}
    ms_index = {"collide": 0, "rows": 1, "pgs": 2, "aba": 4}
    # the last phase times the whole step only (its stage times read 0)
    staged = [t for t in rep["trials"] if not t["ms"][0] == t["ms"][1] == t["ms"][2] == 0.0]
    for kern, fields in KERNEL_FIELDS.items():
        i = ms_index[kern]
        dflt = [t["ms"][i] for t in staged if all(t["shape"][f] == default[f] for f in fields)]
        out["kernels"][kern] = {"tuned_ms": rep["chosen_ms"][kern],
                                "default_ms": float(np.mean(dflt)) if dflt else None}
    out["step_tuned_ms"] = rep["chosen_ms"]["step"]
    # the last phase: whole-step ms per physics step for each partition count (ABA beside
    # collision), for one partition with the ABA kernels in sequence, and for the fused
    # step kernel
    last = [t for t in rep["trials"] if t["ms"][0] == t["ms"][1] == t["ms"][2] == 0.0]
    out["partitions_ms"] = {str(t["shape"]["partitions"]): t["ms"][3] for t in last
                            if t["shape"]["aba_overlap"] and not t["shape"]["fused"]}
    out["aba_in_sequence_ms"] = next((t["ms"][3] for t in last if not t["shape"]["aba_overlap"]), None)
    out["fused_ms"] = next((t["ms"][3] for t in last if t["shape"]["fused"]), None)
    return out


class Workload:
    """One workload on the GPU, advanced to the timed window's first state S0."""

    def __init__(self, cfg, E, rank, dev, warm, mlp, n_control):
        import torch
        from paper_2106_14405_gb300 import Sim
        self.cfg, self.E, self.warm, self.mlp, self.dev = cfg, E, warm, mlp, dev
        self.sub = step_physics(cfg)  # physics steps per benchmark step
        self.b = sg.make_batch(cfg, E, seed_offset=rank_seed_offset(rank, E))
        self.p = sg.params_for(cfg)
        self.p.warm_mode = WARM[warm]
        self.sim = Sim(self.b, self.p, use_graph=True)
        if mlp is not None:
            self.sim.set_mlp(mlp)
        self.walk = None
        if cfg == 5:  # joint targets from a seeded random walk, refreshed every benchmark step (precomputed)
            tg = self.b["joint_target"].copy()
            seq = []
            for k in range(n_control):
                tg = sg.random_walk_targets(self.b, k, tg)
                seq.append(tg.astype(np.float32))
            self.walk = torch.from_numpy(np.stack(seq)).to(dev)
        for k in range(WINDOW_START // self.sub):
            self.control(k)
            self.sim.step(self.sub)
        self.S0 = self.sim.get_state(to_device=True)
        self.S0_host = self.sim.get_state()

    def control(self, k):
        if self.walk is not None:
            self.sim.set_joint_targets(self.walk[k])

    def restore(self):
        self.sim.set_state(self.S0)


def run_timed(wl, args, autotune, world, clocks=True):
    """Tuning and warm-up from S0 (restored after each), then the K timed steps of the
    window; returns the timing record and keeps the window's end state on `wl`."""
    import torch
    import torch.distributed as dist
    sim = wl.sim
    tune = None
    if autotune:
        # trials of one benchmark step each (15 physics steps), so the tuning's rounds
        # sample the window's own course: the drop, then the settling
        tune = tune_summary(sim.launch_shape(), sim.autotune(steps_per_trial=wl.sub, rounds=4))
        wl.restore()
    c0 = WINDOW_START // wl.sub
    sim.set_profiling(False)  # no event nodes in the timed graph (the PGS kernel is timed in its own pass)
    for k in range(args.warmup):
        wl.control(c0 + k)
        sim.step(wl.sub)
    torch.cuda.synchronize()
    wl.restore()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=wl.dev)  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream()
    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    rows_sweeps, nbytes = 0, 0.0
    l0 = sim.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(wl.dev.index or 0) if clocks else None
    for k in range(K):
        flush.zero_()
        ev0[k].record(stream)
        wl.control(c0 + k)
        sim.step(wl.sub)
        ev1[k].record(stream)
        t = sim.totals()
        rows_sweeps += t["row_sweeps"]
        nbytes += pgs_bytes(t, wl.b.n_objects, wl.b.n_joints)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk_rec = clk.stop() if clk else None
    st = sim.stats()
    wl.heaviest = int(np.argmax(st["iters"].astype(np.int64) * np.maximum(st["n_colours"], 1)))
    launches = sim.launch_count() - l0
    total_ms = max_over_ranks(sum(a.elapsed_time(c) for a, c in zip(ev0, ev1)), wl.dev)
    ms_per_step = total_ms / K
    rc, acc, _ = sim.sync()
    wl.S_end = sim.get_state()
    pgs_ms, pgs_launch = pgs_pass(wl, K)
    return {"ms_per_step": ms_per_step, "value": whole_job_rate(world, wl.E, wl.sub, ms_per_step / 1e3),
            "pgs_ms_per_launch": pgs_ms / max(1, pgs_launch), "pgs_ms_per_step": pgs_ms / K,
            "launches": int(launches), "row_sweeps_per_env_step": rows_sweeps / (K * wl.E),
            "pgs_bytes_per_launch": nbytes / K, "clocks": clk_rec, "status": acc, "tune": tune,
            "window": list(timed_window(args.warmup, K, wl.cfg))}


def pgs_pass(wl, K):
    """The PGS kernel's device time over the same window: CUDA event nodes around it in
    the replayed graph (the step then runs unpartitioned, so the kernel is timed alone);
    the window's end state is kept as the timed region left it."""
    import torch
    sim = wl.sim
    end = sim.get_state(to_device=True)
    sim.set_profiling("pgs")
    wl.restore()
    for _ in range(2):
        sim.step(wl.sub)  # graph capture with the events
    torch.cuda.synchronize()
    wl.restore()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=wl.dev)
    c0 = WINDOW_START // wl.sub
    ms_tot, n = 0.0, 0
    for k in range(K):
        flush.zero_()
        wl.control(c0 + k)
        sim.step(wl.sub)
        ms, ln = sim.kernel_times()
        ms_tot += ms["pgs"]
        n += ln["pgs"]
    sim.set_profiling(False)
    sim.set_state(end)
    return ms_tot, n


def stage_pass(wl, K):
    """Per-stage device time over the same window, with events around every kernel."""
    import torch
    sim = wl.sim
    sim.set_profiling(True)
    wl.restore()
    for _ in range(2):
        sim.step(wl.sub)  # graph capture with the events
    torch.cuda.synchronize()
    wl.restore()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=wl.dev)
    c0 = WINDOW_START // wl.sub
    stage = {k: 0.0 for k in STAGES}
    launch = {k: 0 for k in STAGES}
    for k in range(K):
        flush.zero_()
        wl.control(c0 + k)
        sim.step(wl.sub)
        ms, ln = sim.kernel_times()
        for s in STAGES:
            stage[s] += ms[s]
            launch[s] += ln[s]
    sim.set_profiling(False)
    return stage, launch


def mlp_pass(wl, nsteps):
    """The learned warm start's inference kernel over the window's first `nsteps`
    physics steps, one step per call with events around every kernel: its device time
    and the contacts it served in each step, as a tensor-core roofline."""
    sim = wl.sim
    sim.set_params(wl.p)  # the workload's own solver settings (the parity step may have changed them)
    sim.set_profiling(True)
    wl.restore()
    sim.step(1)  # graph capture with the events
    wl.restore()
    ms_tot, rows = 0.0, 0
    for _ in range(nsteps):
        sim.step(1)
        ms, _ = sim.kernel_times()
        ms_tot += ms["mlp"]
        rows += sim.totals()["n_net_rows"]
    sim.set_profiling(False)
    peak, src = bf16_peak()
    achieved = rows * MLP_FLOP_PER_ROW / (ms_tot / 1e3) / 1e12 if ms_tot > 0 else 0.0
    return {"bound": "tensor", "kernel": "mlp (k_mlp_tc)", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_source": src, "rows_per_physics_step": rows / nsteps,
            "flop_per_row": MLP_FLOP_PER_ROW, "kernel_ms_per_physics_step": ms_tot / nsteps,
            "sample": f"physics steps {WINDOW_START}-{WINDOW_START + nsteps}, one per call, CUDA events around the "
                      "kernel, rows from sim_get_stats"}


E2E_PASSES = 3  # timed end-to-end passes over the window (host stalls show in one pass, not in the median)


def e2e_pass(wl, K, world):
    """The same window end to end through the public API with host buffers: joint
    targets host-to-device and the observation device-to-host every step."""
    import torch
    import torch.distributed as dist
    sim = wl.sim
    targets = torch.from_numpy(wl.S0_host["joint_target"].astype(np.float32)).pin_memory().numpy()
    obs_fields = ("obj_pos", "obj_quat", "joint_q", "joint_qd")
    obs = sim._alloc_state(False, pinned=True)
    obs = {k: obs[k] for k in obs_fields}
    sim.set_profiling(False)
    wl.restore()
    for _ in range(2):
        sim.set_joint_targets(targets)
        sim.step(wl.sub)
        sim.get_state(fields=obs_fields, out=obs)
    rates = []
    for _ in range(E2E_PASSES):  # each pass from the window's first state; the median is reported
        wl.restore()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            sim.set_joint_targets(targets)
            sim.step(wl.sub)
            sim.get_state(fields=obs_fields, out=obs)
        torch.cuda.synchronize()
        secs = max_over_ranks(time.perf_counter() - t0, wl.dev)
        rates.append(whole_job_rate(world, wl.E, wl.sub * K, secs))
    return {"value": float(np.median(rates)), "unit": UNIT, "passes": rates,
            "h2d_bytes_per_step": int(targets.nbytes), "d2h_bytes_per_step": int(sum(v.nbytes for v in obs.values()))}


def parity_step(wl):
    """One engine step from the window's end state with the Kahan compensations cleared
    (the oracle starts from the same values); keeps start, result and contact keys."""
    sim = wl.sim
    gs = {k: np.array(v, copy=True) for k, v in wl.S_end.items()}
    gs["obj_pos_comp"][:] = 0
    gs["joint_q_comp"][:] = 0
    if wl.warm == "learned":
        q = sg.params_for(wl.cfg)
        q.warm_mode, q.pgs_tol, q.pgs_max_iters = 2, 1e-6, 1000
        sim.set_params(q)
    sim.set_state(gs)
    sim.step(1)
    sim.sync()
    wl.P_start, wl.P_after, wl.P_contacts = gs, sim.get_state(), sim.contact_keys()


def roofline(flops_per_env_step, E, kernel_ms, fp32, nbytes, hbm, traffic):
    achieved = flops_per_env_step * E / (kernel_ms / 1e3) / 1e12
    gbs = nbytes / (kernel_ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": fp32["tflops"], "unit": "TFLOP/s",
            "frac": achieved / fp32["tflops"], "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "kernel": "pgs", "kernel_ms_per_launch": kernel_ms,
            "kernel_time_source": "CUDA events around the PGS kernel in a pass over the same window (unpartitioned)",
            "algorithmic_flop_per_env_step": flops_per_env_step,
            "peak_source": f"of measured: the library's FP32 FMA probe (sim_fp32_fma_peak), "
                           f"{fp32['ms']:.2f} ms at SM clock {fp32.get('sm_mhz')} MHz",
            "hbm": {"achieved": gbs, "peak": hbm[0], "unit": "GB/s", "frac": gbs / hbm[0],
                    "algorithmic_bytes_per_launch": nbytes, "peak_source": hbm[1]}}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2106_14405_gb300.engine import fp32_fma_peak

    world, rank, local = rank_layout()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    cfg = args.config
    E = args.envs or ENVS.get(cfg, 4096)
    warm = args.warm_start or default_warm_start(cfg)
    n_control = WINDOW_START // step_physics(cfg) + max(args.warmup, args.steps) + 2
    mlp = train_warm_start_network(cfg, pairs=4_000_000, envs=4096, epochs=8)[0] if warm == "learned" else None
    wl = Workload(cfg, E, rank, dev, warm, mlp, n_control)
    if args.shape:
        wl.sim.set_launch_shape(**json.loads(args.shape))
    rec = run_timed(wl, args, autotune=not args.no_autotune and not args.shape, world=world)
    stage_all, launch_all = stage_pass(wl, args.steps)
    e2e = e2e_pass(wl, args.steps, world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    threads = os.cpu_count() or 1
    single = world == 1
    clk = ClockSampler(dev.index or 0)
    tf, pms = fp32_fma_peak(iters=4096, reps=5)
    ck = clk.stop()
    fp32 = {"tflops": tf, "ms": pms, "sm_mhz": ck["sm_mhz"] if ck else None}
    hbm = hbm_peak()
    parity_step(wl)
    cpu = cpu_leg(wl, args.steps, threads, full=True) if single and not args.no_cpu_baseline else None
    roof = None
    if cpu is not None:
        roof = roofline(cpu["counts"]["pgs"], E, rec["pgs_ms_per_launch"], fp32, rec["pgs_bytes_per_launch"], hbm,
                        pgs_traffic(cfg, E))
        roof["oracle_row_sweeps_per_env_step"] = cpu["counts"]["row_sweeps"]
        roof["gpu_row_sweeps_per_env_step"] = rec["row_sweeps_per_env_step"]
        roof["flop_per_row_sweep"] = cpu["counts"]["pgs"] / max(1e-9, cpu["counts"]["row_sweeps"])
        roof["flop_count_sample"] = cpu["count_sample"]
    dom = max(STAGES, key=lambda s: stage_all[s])
    shape = wl.sim.launch_shape()
    wl.sim.close()
    del wl
    torch.cuda.empty_cache()
    extra = {}
    if single:
        for c in [int(x) for x in args.extra_configs.split(",") if x.strip()]:
            if c == cfg:
                continue
            extra[f"workload_{c}"] = run_extra(c, args, dev, threads, fp32, hbm)
    study = None
    if single and not args.no_warm_start_study:
        study = warm_start_study()
    out = {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(cfg, E), "envs_per_gpu": E, "physics_steps_per_step": step_physics(cfg),
                   "physics_step_window": rec["window"], "dt": sg.params_for(cfg).dt,
                   "pgs_sweeps": sg.params_for(cfg).pgs_iters, "warm_start": warm,
                   "l2": "flushed (256 MB write) between timed steps", "graph": True,
                   "tuning": "autotuner and warm-up run from the window's first state, which is restored after each",
                   "launch_shape": shape, "autotune": rec["tune"]},
        "e2e": e2e, "gpu_launches": rec["launches"],
        "stage_ms_per_step": {s: stage_all[s] / args.steps for s in STAGES}, "dominant_stage": dom,
        "stage_ms_source": f"separate pass over the same window ({args.steps} bench steps), events around every "
                           "kernel (L2 flushed between steps)",
        "pgs_ms_per_step_timed": rec["pgs_ms_per_step"], "pgs_row_sweeps_per_env_step": rec["row_sweeps_per_env_step"],
        "roofline": roof, "cpu_baseline": cpu["cpu_baseline"] if cpu else None,
        "parity": cpu["parity"] if cpu else None, "fp32_peak": fp32, "clocks": rec["clocks"],
        "status": rec["status"], "extra_workloads": extra, "warm_start_study": study,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_extra(cfg, args, dev, threads, fp32, hbm):
    """Another workload measured the same way (value, ms per step, PGS roofline, parity)."""
    import torch
    E = ENVS[cfg]
    warm = default_warm_start(cfg)
    t0 = time.perf_counter()
    mlp, train_info = None, None
    if warm == "learned":
        mlp, n, _, cs, ts = train_warm_start_network(cfg, pairs=4_000_000, envs=4096, epochs=8)
        train_info = {"pairs": n, "collect_s": cs, "train_s": ts, "scenes": f"workload {cfg}, seeds disjoint"}
    n_control = WINDOW_START // step_physics(cfg) + max(args.warmup, args.steps) + 2
    wl = Workload(cfg, E, 0, dev, warm, mlp, n_control)
    rec = run_timed(wl, args, autotune=not args.no_autotune, world=1)
    parity_step(wl)
    cpu = cpu_leg(wl, args.steps, threads, full=False) if not args.no_cpu_baseline else None
    out = {"workload": workload_name(cfg, E), "envs": E, "value": rec["value"], "unit": UNIT,
           "ms_per_step": rec["ms_per_step"], "physics_steps_per_step": step_physics(cfg),
           "physics_step_window": rec["window"],
           "dt": wl.p.dt, "warm_start": warm, "network": train_info, "gpu_launches": rec["launches"],
           "status": rec["status"], "clocks": rec["clocks"], "launch_shape": wl.sim.launch_shape(),
           "pgs_ms_per_launch": rec["pgs_ms_per_launch"], "pgs_row_sweeps_per_env_step": rec["row_sweeps_per_env_step"]}
    if warm == "learned":
        out["mlp_roofline"] = mlp_pass(wl, 20)
    if cpu is not None:
        out["roofline"] = roofline(cpu["counts"]["pgs"], E, rec["pgs_ms_per_launch"], fp32,
                                   rec["pgs_bytes_per_launch"], hbm, pgs_traffic(cfg, E))
        out["roofline"]["flop_count_sample"] = cpu["count_sample"]
        out["roofline"]["oracle_row_sweeps_per_env_step"] = cpu["counts"]["row_sweeps"]
        out["parity"] = cpu["parity"]
    out["seconds"] = time.perf_counter() - t0
    wl.sim.close()
    del wl
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    """The oracle timed on the host cores over the same window: advanced to physics
    step WINDOW_START, W warm-up steps from there, the state restored, K timed steps."""
    _, rank, _ = rank_layout()
    if rank != 0:  # under torchrun rank 0 alone times the oracle; the others exit without work
        return
    cfg = args.config
    E = args.envs or ENVS.get(cfg, 4096)
    threads = os.cpu_count() or 1
    warm = args.warm_start or default_warm_start(cfg)
    o = oracle_for(cfg, E, warm)
    o.step(WINDOW_START, threads)
    s0 = o.get_state()
    sub = step_physics(cfg)
    o.step(args.warmup * sub, threads)
    o.set_state(s0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.step(sub, threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = E * sub / (ms / 1e3)
    first, last = timed_window(args.warmup, args.steps, cfg)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(cfg, E), "envs_per_gpu": E, "physics_steps_per_step": sub,
                      "physics_step_window": [first, last], "warm_start": warm},
           "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value, "unit": UNIT,
                            "sample": f"{E} envs, physics steps {first}-{last} of the workload on {threads} host "
                                      f"threads (after {args.warmup * sub} untimed warm-up steps from "
                                      f"step {first}, restored)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
