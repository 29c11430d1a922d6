"""Seeded synthetic scene batches for the batched rigid/articulated physics step.

This module is the one input generator that both the CUDA engine and the CPU
oracle consume.  It only *samples* scene descriptions (shapes, sizes, masses,
initial poses, joint targets) and lays them out as flat CSR arrays; it holds
none of the engine's arithmetic (no inertia tensors, no dynamics, no contact
geometry).  Every random number comes from a counter-based SplitMix64
generator (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output n of the stream with seed s is
mix(s + (n + 1) * 0x9E3779B97F4A7C15), so every environment's draws are
independent of how many environments are generated together.

The scenarios stand in for the paper's benchmark scenes (a Fetch-like mobile
manipulator in a furnished apartment with clutter on receptacles, doors and
drawers, Sec. 4.4 "Benchmarking" and Sec. 5.1 "Agent embodiment"), whose assets
are not available here; sizes follow the five workload descriptions:

  1  64 fixed 7-DoF arms, no contacts                      (make_batch(1))
  2  4096 mobile manipulators + 10 dropped objects + 20 static boxes
  3  16384 uneven envs: 2..40 objects, 0..6 doors/drawers
  4  scenes of workload 2 on held-out seeds (learned warm start)
  5  65536 envs, 30 objects, 4 doors/drawers, dt = 1/240
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SHAPE_SPHERE = 0
SHAPE_BOX = 1
JOINT_REVOLUTE = 0
JOINT_PRISMATIC = 1

# Layout constants of the synthetic apartment (metres).
STATIC_GRID_X = (-2.4, -1.2, 0.0, 1.2, 2.4)
STATIC_GRID_Y = (-2.4, -1.2, 1.2, 2.4)
RECEPTACLE_SLOTS = ((-2.4, 0.0), (-1.2, 0.0), (1.2, 0.0), (2.4, 0.0), (-3.6, 0.0), (3.6, 0.0))
ROBOT_MOUNT_Z = 0.8
ROBOT_BASE_HALF = (0.25, 0.25, 0.2)
ARM_LINK_HALF_WIDTH = 0.03
FINGER_HALF = (0.03, 0.01, 0.01)
FINGER_MASS = 0.05


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class CounterRng:
    """Per-environment counter-based streams, vectorised over environments."""

    def __init__(self, seeds: np.ndarray):
        self.seeds = np.asarray(seeds, dtype=np.uint64)
        self.counter = 0

    def raw(self, k: int) -> np.ndarray:
        n = np.arange(self.counter + 1, self.counter + 1 + k, dtype=np.uint64)
        self.counter += k
        with np.errstate(over="ignore"):
            x = self.seeds[:, None] + n[None, :] * GAMMA
        return splitmix64_mix(x)

    def uniform(self, k: int, lo=0.0, hi=1.0) -> np.ndarray:
        """[E, k] doubles in [lo, hi)."""
        u = (self.raw(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, k: int, lo: int, hi_inclusive: int) -> np.ndarray:
        u = self.uniform(k)
        return (lo + np.floor(u * (hi_inclusive - lo + 1))).astype(np.int64).clip(lo, hi_inclusive)

    def normal(self, k: int) -> np.ndarray:
        """Box-Muller normal draws (two uniforms per draw)."""
        u1 = self.uniform(k)
        u2 = self.uniform(k)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _quat_yaw(yaw):
    yaw = np.asarray(yaw, dtype=np.float64)
    return np.stack([np.cos(yaw / 2), np.zeros_like(yaw), np.zeros_like(yaw), np.sin(yaw / 2)], -1)


def _quat_uniform(u1, u2, u3):
    """Uniformly distributed unit quaternion (w, x, y, z) from three uniforms (Shoemake 1992)."""
    a = np.sqrt(1 - u1)
    b = np.sqrt(u1)
    x = a * np.sin(2 * math.pi * u2)
    y = a * np.cos(2 * math.pi * u2)
    z = b * np.sin(2 * math.pi * u3)
    w = b * np.cos(2 * math.pi * u3)
    return np.stack([w, x, y, z], -1)


@dataclass
class SimParams:
    """Step parameters shared by both engines (all SI units)."""

    dt: float = 1.0 / 120.0
    gravity: tuple = (0.0, 0.0, -9.81)
    pgs_iters: int = 10          # sweeps when pgs_tol == 0
    pgs_tol: float = 0.0         # > 0: iterate until relative residual <= tol
    pgs_max_iters: int = 1000
    baumgarte: float = 0.2
    slop: float = 0.001
    margin: float = 0.02         # contact generation distance; AABBs fattened by margin / 2
    rest_thresh: float = 0.5     # restitution applies below -rest_thresh approach speed
    sleep_lin: float = 0.05
    sleep_ang: float = 0.05
    sleep_steps: int = 60        # round(0.5 s / dt)
    sleep_enabled: int = 1
    warm_mode: int = 1           # 0 cold, 1 prior frame, 2 learned
    plane_mu: float = 0.5
    lambda_floor: float = 1e-4 * 9.81 / 120.0
    match_dist: float = 0.01
    max_contacts: int = 256
    fp64_cond: float = 1e4       # GPU only: recompute M^-1 in FP64 above this D-ratio
    force_limit: float = 5000.0  # N; accumulated robot contact force that flags an env (<= 0: off)
    motor_mode: int = 0          # 1: robot joints driven by impulse-capped motor rows instead of the implicit PD
    motor_kp: float = 0.3        # motor position gain (target rate kp (q_target - q) / dt)
    motor_max_impulse: float = 10.0  # N s per step and joint

    def with_dt(self, dt: float) -> "SimParams":
        p = SimParams(**self.__dict__)
        p.dt = dt
        p.sleep_steps = int(round(0.5 / dt))
        p.lambda_floor = 1e-4 * 9.81 * dt
        return p


@dataclass
class Batch:
    """Flat CSR scene description; every float array is float64, every index int32."""

    n_envs: int
    arrays: dict = field(default_factory=dict)

    def __getitem__(self, k):
        return self.arrays[k]

    def __setitem__(self, k, v):
        self.arrays[k] = v

    @property
    def n_objects(self):
        return int(self.arrays["obj_off"][-1])

    @property
    def n_joints(self):
        return int(self.arrays["joint_off"][-1])

    @property
    def n_arts(self):
        return int(self.arrays["art_off"][-1])

    def subset(self, envs) -> "Batch":
        """The batch restricted to the given environments (envs never interact)."""
        envs = np.asarray(envs, dtype=np.int64)
        a = self.arrays
        out = {}

        def csr_take(off, per_item_keys):
            starts, ends = off[envs], off[envs + 1]
            idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if len(envs) else np.zeros(0, np.int64)
            idx = idx.astype(np.int64)
            new_off = np.zeros(len(envs) + 1, np.int32)
            new_off[1:] = np.cumsum(ends - starts)
            for k in per_item_keys:
                out[k] = a[k][idx].copy()
            return idx, new_off

        _, out["obj_off"] = csr_take(a["obj_off"], [k for k in a if k.startswith("obj_") and k != "obj_off"])
        _, out["stat_off"] = csr_take(a["stat_off"], [k for k in a if k.startswith("stat_") and k != "stat_off"])
        art_idx, out["art_off"] = csr_take(a["art_off"], [k for k in a if k.startswith("art_") and k not in ("art_off",)])
        joff = a["joint_off"]
        jidx = np.concatenate([np.arange(joff[i], joff[i + 1]) for i in art_idx]) if len(art_idx) else np.zeros(0, np.int64)
        jidx = jidx.astype(np.int64)
        new_joff = np.zeros(len(art_idx) + 1, np.int32)
        new_joff[1:] = np.cumsum(joff[art_idx + 1] - joff[art_idx])
        out["joint_off"] = new_joff
        for k in a:
            if k.startswith("joint_") and k != "joint_off":
                out[k] = a[k][jidx].copy()
        for k in a:
            if k.startswith("env_"):
                out[k] = a[k][envs].copy()
        return Batch(len(envs), out)


def _csr(counts):
    off = np.zeros(len(counts) + 1, np.int32)
    off[1:] = np.cumsum(counts)
    return off


def _arm_chain(rng: CounterRng, E: int, base_z: float, with_fingers: bool, with_limits: bool):
    """Per-env 7-DoF revolute arm (+ optional 2 prismatic fingers) as joint arrays [E, nj]."""
    lengths = rng.uniform(7, 0.1, 0.4)
    masses = rng.uniform(7, 0.5, 3.0)
    nj = 9 if with_fingers else 7
    J = {}
    J["parent"] = np.tile(np.array([-1, 0, 1, 2, 3, 4, 5] + ([6, 6] if with_fingers else []), np.int32), (E, 1))
    J["type"] = np.tile(np.array([JOINT_REVOLUTE] * 7 + ([JOINT_PRISMATIC] * 2 if with_fingers else []), np.int32), (E, 1))
    axes = np.zeros((E, nj, 3))
    for i in range(7):
        axes[:, i, 2 if i % 2 == 0 else 1] = 1.0
    if with_fingers:
        axes[:, 7, 1] = 1.0
        axes[:, 8, 1] = -1.0
    J["axis"] = axes
    origin = np.zeros((E, nj, 3))
    origin[:, 0, 2] = base_z
    origin[:, 1:7, 0] = lengths[:, 0:6]
    if with_fingers:
        origin[:, 7, 0] = lengths[:, 6]
        origin[:, 8, 0] = lengths[:, 6]
    J["origin_pos"] = origin
    oq = np.zeros((E, nj, 4))
    oq[..., 0] = 1.0
    J["origin_quat"] = oq
    com = np.zeros((E, nj, 3))
    com[:, 0:7, 0] = lengths / 2
    half = np.zeros((E, nj, 3))
    half[:, 0:7, 0] = lengths / 2
    half[:, 0:7, 1] = ARM_LINK_HALF_WIDTH
    half[:, 0:7, 2] = ARM_LINK_HALF_WIDTH
    mass = np.zeros((E, nj))
    mass[:, 0:7] = masses
    if with_fingers:
        com[:, 7:9, 0] = FINGER_HALF[0]
        half[:, 7:9, :] = FINGER_HALF
        mass[:, 7:9] = FINGER_MASS
    J["com"] = com
    J["half"] = half
    J["mass"] = mass
    lo = np.zeros((E, nj))
    hi = np.zeros((E, nj))
    has = np.zeros((E, nj), np.int32)
    if with_limits:
        lo[:, 0:7] = -2.5
        hi[:, 0:7] = 2.5
        has[:, 0:7] = 1
        if with_fingers:
            lo[:, 7:9] = 0.0
            hi[:, 7:9] = 0.05
            has[:, 7:9] = 1
    J["lo"], J["hi"], J["has_limit"] = lo, hi, has
    J["kp"] = np.full((E, nj), 100.0)
    J["kd"] = np.full((E, nj), 10.0)
    J["mu"] = np.full((E, nj), 0.5)
    J["q0"] = np.zeros((E, nj))
    if with_limits:
        # mobile manipulator: start with the arm pointing straight up (joint 2 about y at -pi/2),
        # clear of the receptacles around the robot
        J["q0"][:, 1] = -0.5 * math.pi
    J["qd0"] = np.zeros((E, nj))
    tgt = np.zeros((E, nj))
    tgt[:, 0:7] = rng.uniform(7, -1.0, 1.0)
    if with_fingers:
        tgt[:, 7:9] = rng.uniform(2, 0.0, 0.05)
    J["target"] = tgt
    return J


def _receptacle_joints(rng: CounterRng, E: int, n_rec: np.ndarray):
    """Doors (revolute about z at the panel edge, [0, 1.6] rad) and drawers (prismatic, [0, 0.4] m)
    per receptacle slot, [E, 6] draws: kind (0 door, 1 drawer), mass U(2, 10), initial position
    fraction U(0, 0.5) of the range, initial rate U(-0.5, 0.5) (drawers scaled by 0.2)."""
    R = len(RECEPTACLE_SLOTS)
    kind = (rng.uniform(R) < 0.5).astype(np.int32)
    mass = rng.uniform(R, 2.0, 10.0)
    qfrac = rng.uniform(R, 0.0, 0.5)
    qd0 = rng.uniform(R, -0.5, 0.5)
    return kind, mass, qfrac, qd0


def _spawn_objects(rng: CounterRng, E: int, n_obj: np.ndarray, stat_pos, stat_half, n_max: int):
    """Objects dropped from U(0, 0.3) m above a random static receptacle's top; bounding
    spheres never overlap at t = 0 (rejection sampling, 64 attempts, then stacked higher)."""
    shape_u = rng.uniform(n_max)
    is_box = shape_u < 0.5
    box_half = rng.uniform(3 * n_max, 0.03, 0.15).reshape(E, n_max, 3)
    radius = rng.uniform(n_max, 0.03, 0.1)
    mass = rng.uniform(n_max, 0.1, 1.0)
    qu = rng.uniform(3 * n_max).reshape(E, n_max, 3)
    half = np.where(is_box[..., None], box_half, np.stack([radius, radius, radius], -1))
    bound = np.where(is_box, np.linalg.norm(box_half, axis=-1), radius)
    pos = np.zeros((E, n_max, 3))
    placed = np.zeros((E, n_max), bool)
    n_stat = stat_pos.shape[1]
    for j in range(n_max):
        need = n_obj > j
        done = ~need
        for attempt in range(64):
            u = rng.uniform(4)  # drawn for every env so each env's stream is independent of the others
            todo = np.nonzero(~done)[0]
            ut = u[todo]
            r = np.minimum((ut[:, 0] * n_stat).astype(np.int64), n_stat - 1)
            sp = stat_pos[todo, r]
            sh = stat_half[todo, r]
            top = sp[:, 2] + sh[:, 2]
            bj = bound[todo, j]
            mx = np.maximum(sh[:, 0] - bj, 0.0)
            my = np.maximum(sh[:, 1] - bj, 0.0)
            cand = np.stack([sp[:, 0] + (2 * ut[:, 1] - 1) * mx,
                             sp[:, 1] + (2 * ut[:, 2] - 1) * my,
                             top + bj + 0.3 * ut[:, 3]], -1)
            if attempt == 63:
                cand[:, 2] += 0.6 + 0.6 * j  # give up on this receptacle layout: stack higher
                ok = np.ones(len(todo), bool)
            elif j > 0:
                dist = np.sqrt(((cand[:, None, :] - pos[todo, :j, :]) ** 2).sum(-1))
                clash = placed[todo, :j] & (dist < bj[:, None] + bound[todo, :j] + 0.005)
                ok = ~clash.any(1)
            else:
                ok = np.ones(len(todo), bool)
            take = todo[ok]
            pos[take, j] = cand[ok]
            placed[take, j] = True
            done[take] = True
            if done.all():
                break
    quat = _quat_uniform(qu[..., 0], qu[..., 1], qu[..., 2])
    return is_box, half, mass, pos, quat


def make_batch(config: int, n_envs: int | None = None, seed_offset: int = 0) -> Batch:
    """Synthetic batch for workload `config` (1..5); env i uses seed 1000*config + seed_offset + i."""
    defaults = {1: 64, 2: 4096, 3: 16384, 4: 4096, 5: 65536}
    E = defaults[config] if n_envs is None else int(n_envs)
    seeds = (1000 * config + seed_offset + np.arange(E)).astype(np.uint64)
    rng = CounterRng(seeds)
    A = {}
    if config == 1:
        J = _arm_chain(rng, E, 0.0, with_fingers=False, with_limits=False)
        nj = 7
        A["obj_off"] = _csr(np.zeros(E, np.int64))
        for k, w in (("obj_shape", 0), ("obj_half", 3), ("obj_mass", 0), ("obj_mu", 0), ("obj_rest", 0),
                     ("obj_pos", 3), ("obj_quat", 4), ("obj_vel", 3), ("obj_omega", 3)):
            A[k] = np.zeros((0, w) if w else (0,), np.int32 if k == "obj_shape" else np.float64)
        A["stat_off"] = _csr(np.zeros(E, np.int64))
        A["stat_pos"] = np.zeros((0, 3))
        A["stat_quat"] = np.zeros((0, 4))
        A["stat_half"] = np.zeros((0, 3))
        A["stat_mu"] = np.zeros(0)
        A["art_off"] = _csr(np.ones(E, np.int64))
        A["joint_off"] = _csr(np.full(E, nj))
        A["art_base_pos"] = np.tile([0.0, 0.0, 3.0], (E, 1))
        A["art_base_quat"] = np.tile([1.0, 0.0, 0.0, 0.0], (E, 1))
        A["art_has_base_coll"] = np.zeros(E, np.int32)
        A["art_base_coll_off"] = np.zeros((E, 3))
        A["art_base_coll_half"] = np.zeros((E, 3))
        A["art_kinematic"] = np.zeros(E, np.int32)
        for k, v in J.items():
            A["joint_" + k] = v.reshape((E * nj,) + v.shape[2:]).astype(v.dtype)
        A["env_plane"] = np.zeros(E, np.int32)
        return _finish(Batch(E, A))

    # Workloads 2..5: mobile manipulator + 20 static boxes + free objects (+ receptacles).
    if config in (2, 4):
        n_obj = np.full(E, 10)
        n_rec = np.zeros(E, np.int64)
    elif config == 3:
        n_obj = rng.integers(1, 2, 40)[:, 0]
        n_rec = rng.integers(1, 0, 6)[:, 0]
    else:
        n_obj = np.full(E, 30)
        n_rec = np.full(E, 4)
    n_max = int(n_obj.max()) if E else 0

    # Static receptacle boxes: 5 x 4 grid with 1.2 m pitch (row y = 0 left for the robot).
    ns = len(STATIC_GRID_X) * len(STATIC_GRID_Y)
    hxy = rng.uniform(2 * ns, 0.2, 0.5).reshape(E, ns, 2)
    top = rng.uniform(ns, 0.4, 0.9)
    gx, gy = np.meshgrid(STATIC_GRID_X, STATIC_GRID_Y, indexing="ij")
    stat_pos = np.stack([np.broadcast_to(gx.ravel(), (E, ns)), np.broadcast_to(gy.ravel(), (E, ns)), top / 2], -1)
    stat_half = np.concatenate([hxy, (top / 2)[..., None]], -1)

    robot = _arm_chain(rng, E, ROBOT_MOUNT_Z, with_fingers=True, with_limits=True)
    yaw = rng.uniform(1, -math.pi, math.pi)[:, 0]
    recs = _receptacle_joints(rng, E, n_rec)
    is_box, ohalf, omass, opos, oquat = _spawn_objects(rng, E, n_obj, stat_pos, stat_half, n_max)

    # Flatten objects.
    mask = np.arange(n_max)[None, :] < n_obj[:, None]
    A["obj_off"] = _csr(n_obj)
    A["obj_shape"] = np.where(is_box, SHAPE_BOX, SHAPE_SPHERE).astype(np.int32)[mask]
    A["obj_half"] = ohalf[mask]
    A["obj_mass"] = omass[mask]
    A["obj_mu"] = np.full(int(mask.sum()), 0.5)
    A["obj_rest"] = np.zeros(int(mask.sum()))
    A["obj_pos"] = opos[mask]
    A["obj_quat"] = oquat[mask]
    A["obj_vel"] = np.zeros((int(mask.sum()), 3))
    A["obj_omega"] = np.zeros((int(mask.sum()), 3))
    A["stat_off"] = _csr(np.full(E, ns))
    A["stat_pos"] = stat_pos.reshape(-1, 3)
    A["stat_quat"] = np.tile([1.0, 0.0, 0.0, 0.0], (E * ns, 1))
    A["stat_half"] = stat_half.reshape(-1, 3)
    A["stat_mu"] = np.full(E * ns, 0.5)

    # Articulations: the robot (9 joints, kinematic planar base) then 1-DoF receptacles,
    # assembled as [E, 1 + 6] articulation slots and [E, 9 + 6] joint slots, masked.
    R = len(RECEPTACLE_SLOTS)
    n_art = 1 + n_rec
    A["art_off"] = _csr(n_art)
    rk, rmass, rq, rqd = recs
    slot_ok = np.arange(R)[None, :] < n_rec[:, None]            # [E, R]
    art_ok = np.concatenate([np.ones((E, 1), bool), slot_ok], 1)
    door = rk == 0
    sx = np.array([s_[0] for s_ in RECEPTACLE_SLOTS])[None, :].repeat(E, 0)
    sy = np.array([s_[1] for s_ in RECEPTACLE_SLOTS])[None, :].repeat(E, 0)
    rbase = np.stack([sx, np.where(door, sy - 0.3, sy), np.where(door, 0.45, 0.5)], -1)
    base_pos = np.concatenate([np.zeros((E, 1, 3)), rbase], 1)
    base_quat = np.concatenate([_quat_yaw(yaw)[:, None, :], np.tile([1.0, 0, 0, 0], (E, R, 1))], 1)
    has_bc = np.concatenate([np.ones((E, 1), np.int32), np.zeros((E, R), np.int32)], 1)
    bc_off = np.zeros((E, 1 + R, 3))
    bc_off[:, 0, 2] = ROBOT_BASE_HALF[2]
    bc_half = np.zeros((E, 1 + R, 3))
    bc_half[:, 0] = ROBOT_BASE_HALF
    kin = np.concatenate([np.ones((E, 1), np.int32), np.zeros((E, R), np.int32)], 1)
    A["art_base_pos"] = base_pos[art_ok]
    A["art_base_quat"] = base_quat[art_ok]
    A["art_has_base_coll"] = has_bc[art_ok]
    A["art_base_coll_off"] = bc_off[art_ok]
    A["art_base_coll_half"] = bc_half[art_ok]
    A["art_kinematic"] = kin[art_ok]
    A["joint_off"] = _csr(np.where(art_ok, np.where(np.arange(1 + R)[None, :] == 0, 9, 1), 0)[art_ok])
    # receptacle joint fields [E, R, ...]
    rj = {
        "parent": np.full((E, R), -1, np.int32),
        "type": np.where(door, JOINT_REVOLUTE, JOINT_PRISMATIC).astype(np.int32),
        "axis": np.where(door[..., None], np.array([0.0, 0, 1]), np.array([1.0, 0, 0])),
        "origin_pos": np.zeros((E, R, 3)),
        "origin_quat": np.tile([1.0, 0, 0, 0], (E, R, 1)),
        "com": np.where(door[..., None], np.array([0.0, 0.3, 0.0]), np.array([0.0, 0.0, 0.0])),
        "half": np.where(door[..., None], np.array([0.02, 0.3, 0.4]), np.array([0.25, 0.2, 0.1])),
        "mass": rmass,
        "lo": np.zeros((E, R)),
        "hi": np.where(door, 1.6, 0.4),
        "has_limit": np.ones((E, R), np.int32),
        "kp": np.zeros((E, R)),
        "kd": np.zeros((E, R)),
        "mu": np.full((E, R), 0.5),
        "q0": rq * np.where(door, 1.6, 0.4),
        "qd0": rqd * np.where(door, 1.0, 0.2),
        "target": np.zeros((E, R)),
    }
    joint_ok = np.concatenate([np.ones((E, 9), bool), slot_ok], 1)
    for k in robot:
        v = np.concatenate([robot[k], rj[k]], 1)
        A["joint_" + k] = v[joint_ok]
    A["env_plane"] = np.ones(E, np.int32)
    return _finish(Batch(E, A))


def _finish(b: Batch) -> Batch:
    for k, v in list(b.arrays.items()):
        if v.dtype.kind in "iu":
            b.arrays[k] = np.ascontiguousarray(v, dtype=np.int32)
        else:
            b.arrays[k] = np.ascontiguousarray(v, dtype=np.float64)
    return b


def params_for(config: int) -> SimParams:
    """Step parameters of each workload."""
    p = SimParams()
    if config == 1:
        p.sleep_enabled = 0
    if config == 4:
        p.pgs_tol = 1e-6
        p.pgs_max_iters = 1000
    if config == 5:
        p = p.with_dt(1.0 / 240.0)
    return p


def robot_joint_index(b: Batch) -> np.ndarray:
    """Global joint indices of every env's robot (articulation 0), [E, 9] (or [E, 7])."""
    first = b["joint_off"][b["art_off"][:-1]]
    n = b["joint_off"][b["art_off"][:-1] + 1] - first
    return first[:, None] + np.arange(int(n.max()))[None, :]


def random_walk_targets(b: Batch, step: int, prev: np.ndarray, sigma: float = 0.05, seed: int = 5) -> np.ndarray:
    """Joint targets after one seeded random-walk control step: N(0, sigma) rad per arm joint,
    clipped to the joint limits; non-robot joints keep their targets. `prev` is [n_joints]."""
    out = prev.copy()
    E = b.n_envs
    idx = robot_joint_index(b)
    seeds = (1_000_000 * seed + np.arange(E)).astype(np.uint64)
    rng = CounterRng(seeds)
    rng.counter = 4 * idx.shape[1] * step
    d = rng.normal(idx.shape[1]) * sigma
    lo = b["joint_lo"][idx]
    hi = b["joint_hi"][idx]
    has = b["joint_has_limit"][idx] > 0
    new = out[idx] + d
    new = np.where(has, np.clip(new, lo, hi), new)
    out[idx] = new
    return out


def custom_batch(envs) -> Batch:
    """Hand-written scenes for tests.  `envs` is a list of dicts with optional keys
    objects  : list of dict(shape, half, mass, mu=0.5, rest=0, pos, quat=(1,0,0,0), vel=0, omega=0)
    statics  : list of dict(pos, half, quat=(1,0,0,0), mu=0.5)
    arts     : list of dict(base_pos, base_quat=(1,0,0,0), base_coll=None|(off, half), kinematic=0,
                            joints=[dict(parent, type, axis, origin_pos, origin_quat, com, half, mass,
                                         lo=0, hi=0, has_limit=0, kp=0, kd=0, mu=0.5, q0=0, qd0=0, target=0)])
    plane    : bool (ground plane z = 0)."""
    A = {k: [] for k in ("obj_shape", "obj_half", "obj_mass", "obj_mu", "obj_rest", "obj_pos", "obj_quat",
                         "obj_vel", "obj_omega", "stat_pos", "stat_quat", "stat_half", "stat_mu", "art_base_pos",
                         "art_base_quat", "art_has_base_coll", "art_base_coll_off", "art_base_coll_half",
                         "art_kinematic", "joint_parent", "joint_type", "joint_axis", "joint_origin_pos",
                         "joint_origin_quat", "joint_com", "joint_half", "joint_mass", "joint_lo", "joint_hi",
                         "joint_has_limit", "joint_kp", "joint_kd", "joint_mu", "joint_q0", "joint_qd0",
                         "joint_target", "env_plane")}
    n_obj, n_stat, n_art, n_j = [], [], [], []
    for env in envs:
        objs = env.get("objects", [])
        n_obj.append(len(objs))
        for o in objs:
            A["obj_shape"].append(o["shape"])
            h = o["half"]
            A["obj_half"].append((h, h, h) if np.isscalar(h) else tuple(h))
            A["obj_mass"].append(o["mass"])
            A["obj_mu"].append(o.get("mu", 0.5))
            A["obj_rest"].append(o.get("rest", 0.0))
            A["obj_pos"].append(tuple(o["pos"]))
            A["obj_quat"].append(tuple(o.get("quat", (1.0, 0.0, 0.0, 0.0))))
            A["obj_vel"].append(tuple(o.get("vel", (0.0, 0.0, 0.0))))
            A["obj_omega"].append(tuple(o.get("omega", (0.0, 0.0, 0.0))))
        sts = env.get("statics", [])
        n_stat.append(len(sts))
        for s in sts:
            A["stat_pos"].append(tuple(s["pos"]))
            A["stat_quat"].append(tuple(s.get("quat", (1.0, 0.0, 0.0, 0.0))))
            A["stat_half"].append(tuple(s["half"]))
            A["stat_mu"].append(s.get("mu", 0.5))
        arts = env.get("arts", [])
        n_art.append(len(arts))
        for a in arts:
            A["art_base_pos"].append(tuple(a["base_pos"]))
            A["art_base_quat"].append(tuple(a.get("base_quat", (1.0, 0.0, 0.0, 0.0))))
            bc = a.get("base_coll")
            A["art_has_base_coll"].append(0 if bc is None else 1)
            A["art_base_coll_off"].append((0.0, 0.0, 0.0) if bc is None else tuple(bc[0]))
            A["art_base_coll_half"].append((0.0, 0.0, 0.0) if bc is None else tuple(bc[1]))
            A["art_kinematic"].append(a.get("kinematic", 0))
            n_j.append(len(a["joints"]))
            for j in a["joints"]:
                A["joint_parent"].append(j["parent"])
                A["joint_type"].append(j["type"])
                A["joint_axis"].append(tuple(j["axis"]))
                A["joint_origin_pos"].append(tuple(j.get("origin_pos", (0.0, 0.0, 0.0))))
                A["joint_origin_quat"].append(tuple(j.get("origin_quat", (1.0, 0.0, 0.0, 0.0))))
                A["joint_com"].append(tuple(j["com"]))
                A["joint_half"].append(tuple(j["half"]))
                A["joint_mass"].append(j["mass"])
                for k, dflt in (("lo", 0.0), ("hi", 0.0), ("has_limit", 0), ("kp", 0.0), ("kd", 0.0),
                                ("mu", 0.5), ("q0", 0.0), ("qd0", 0.0), ("target", 0.0)):
                    A["joint_" + k].append(j.get(k, dflt))
        A["env_plane"].append(1 if env.get("plane", True) else 0)
    widths = {"obj_half": 3, "obj_pos": 3, "obj_quat": 4, "obj_vel": 3, "obj_omega": 3, "stat_pos": 3,
              "stat_quat": 4, "stat_half": 3, "art_base_pos": 3, "art_base_quat": 4, "art_base_coll_off": 3,
              "art_base_coll_half": 3, "joint_axis": 3, "joint_origin_pos": 3, "joint_origin_quat": 4,
              "joint_com": 3, "joint_half": 3}
    ints = {"obj_shape", "art_has_base_coll", "art_kinematic", "joint_parent", "joint_type", "joint_has_limit",
            "env_plane"}
    out = {}
    for k, v in A.items():
        w = widths.get(k)
        arr = np.array(v, dtype=np.int32 if k in ints else np.float64)
        if w is not None:
            arr = arr.reshape(-1, w)
        out[k] = arr
    out["obj_off"] = _csr(np.array(n_obj, np.int64))
    out["stat_off"] = _csr(np.array(n_stat, np.int64))
    out["art_off"] = _csr(np.array(n_art, np.int64))
    out["joint_off"] = _csr(np.array(n_j, np.int64))
    return _finish(Batch(len(envs), out))


def mlp_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the 32-128-128-128-3 warm-start network in the flat
    layout W1[128][32] b1 W2[128][128] b2 W3[128][128] b3 W4[3][128] b4 (He normal weights,
    zero biases).  Both the GPU trainer and the FP64 reference start from these."""
    rng = CounterRng(np.array([7_000_000 + seed], np.uint64))
    parts = []
    for nin, nout in ((32, 128), (128, 128), (128, 128), (128, 3)):
        parts.append(rng.normal(nout * nin)[0] * np.sqrt(2.0 / nin))
        parts.append(np.zeros(nout))
    return np.concatenate(parts)
