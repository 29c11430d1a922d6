"""Learned PGS warm start: dataset logging and training through the C ABI.

The network predicts, per contact, the correction from the prior-frame impulses
to the converged impulses (normal, two friction), in units of the contact's
impulse unit m_eff,n (|g| dt + |v_rel|), from 32 contact features (which include
the prior-frame impulses and the relative velocity before the solve).  The
deployed warm start (sim_set_mlp, warm_mode 2) uses it for the contacts without
a prior-frame match and for the matched ones moving faster than 4 |g| dt
relative to each other; the others keep the prior impulse.  Every computation
runs in the library's kernels: logging in the simulator step (only converged
solves, finite targets), row selection, target clipping and feature statistics
in the trainer's data-preparation calls, forward/backward/Adam in the trainer;
this module only moves arguments and orders the minibatches.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N
from .engine import Sim

NPARAM = 128 * 32 + 128 + 2 * (128 * 128 + 128) + 3 * 128 + 3
LEARN_GATE = 4.0  # matched contacts served by the network: |v_rel| > LEARN_GATE |g| dt


def _p(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


class Trainer:
    """Warm-start network trainer on the current CUDA device."""

    def __init__(self, init_params, batch: int, feat_mean=None, feat_std=None, stream=None):
        self.lib = N.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p = np.ascontiguousarray(init_params, np.float32)
        assert p.size == NPARAM
        mean = None if feat_mean is None else np.ascontiguousarray(feat_mean, np.float32)
        std = None if feat_std is None else np.ascontiguousarray(feat_std, np.float32)
        h = C.c_void_p()
        N.check(self.lib.mlp_train_create(p.ctypes.data_as(C.c_void_p), 0, int(batch),
                                          None if mean is None else mean.ctypes.data_as(C.c_void_p),
                                          None if std is None else std.ctypes.data_as(C.c_void_p),
                                          C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.batch = batch

    def close(self):
        if getattr(self, "h", None):
            self.lib.mlp_train_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, X: torch.Tensor, T: torch.Tensor, lr: float, want_loss: bool = False):
        loss = C.c_float(0.0)
        N.check(self.lib.mlp_train_step(self.h, _p(X), _p(T), int(X.shape[0]), float(lr),
                                        C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def loss_grad(self, X: torch.Tensor, T: torch.Tensor):
        g = torch.empty(NPARAM, dtype=torch.float32, device="cuda")
        loss = C.c_float(0.0)
        N.check(self.lib.mlp_loss_grad(self.h, _p(X), _p(T), int(X.shape[0]), _p(g), C.byref(loss)))
        return float(loss.value), g

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        Y = torch.empty((X.shape[0], 3), dtype=torch.float32, device="cuda")
        N.check(self.lib.mlp_forward(self.h, _p(X), int(X.shape[0]), _p(Y)))
        return Y

    def params(self) -> np.ndarray:
        out = np.zeros(NPARAM, np.float32)
        N.check(self.lib.mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p), 0))
        return out


def select_rows(X: torch.Tensor, T: torch.Tensor, only_used: bool, gate_speed: float, clip: float = 10.0):
    """The training rows (mlp_select_rows): finite targets, with `only_used` just the rows
    the in-step warm start serves, targets clipped; device tensors in, device tensors out."""
    lib = N.load()
    X = X.contiguous().float()
    T = T.contiguous().float()
    Xo, To = torch.empty_like(X), torch.empty_like(T)
    n = C.c_int(0)
    st = torch.cuda.current_stream()
    N.check(lib.mlp_select_rows(_p(X), _p(T), int(X.shape[0]), int(only_used), float(gate_speed), float(clip),
                                _p(Xo), _p(To), C.byref(n), C.c_void_p(st.cuda_stream)))
    return Xo[:n.value], To[:n.value]


def feature_stats(X: torch.Tensor):
    """Per-feature mean and standard deviation (mlp_feature_stats), host arrays."""
    lib = N.load()
    X = X.contiguous().float()
    mean, std = np.zeros(32, np.float32), np.zeros(32, np.float32)
    st = torch.cuda.current_stream()
    N.check(lib.mlp_feature_stats(_p(X), int(X.shape[0]), mean.ctypes.data_as(C.c_void_p),
                                  std.ctypes.data_as(C.c_void_p), 0, C.c_void_p(st.cuda_stream)))
    return mean, std


def collect(batch, params, steps: int, warm_steps: int = 0, cap_per_step: int = 1 << 20, device: bool = False):
    """Run the plain solver (prior-frame warm start) to the params' residual target and
    return the logged (features, normalised impulse corrections) of every step: the
    library logs the contacts of the environments whose solve converged, with finite
    targets.  Host arrays, or device tensors with `device`."""
    sim = Sim(batch, params, use_graph=False, log_features=True)
    if warm_steps:
        sim.step(warm_steps)
    feats, lams = [], []
    for _ in range(steps):
        sim.step(1)
        f, l, n = sim.log_contacts(cap_per_step)
        sim.sync()
        feats.append(f.clone() if device else f.cpu().numpy())
        lams.append(l.clone() if device else l.cpu().numpy())
    sim.close()
    if device:
        return torch.cat(feats), torch.cat(lams)
    return np.concatenate(feats), np.concatenate(lams)


def train(X, T, init_params, epochs: int = 3, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          clip: float = 10.0, only_used: bool = False, gate_speed: float = 4.0 * 9.81 / 120.0):
    """Adam on minibatches of a fixed seeded permutation of the training rows: the
    logged rows (every logged contact, or with `only_used` just those the deployed
    warm start serves, selected by the library with `gate_speed` = 4 |g| dt), targets
    clipped to [-clip, clip] by the library, inputs normalised by the library's
    feature statistics; returns (params for raw features, list of per-epoch mean
    losses).  X, T: host arrays or device tensors."""
    Xd = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X, np.float32))
    Td = T if isinstance(T, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(T, np.float32))
    Xd, Td = select_rows(Xd.cuda(), Td.cuda(), only_used, gate_speed, clip)
    mean, std = feature_stats(Xd)
    tr = Trainer(init_params, batch, mean, std)
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    perm = torch.randperm(Xd.shape[0], generator=g).to(Xd.device)
    Xd, Td = Xd[perm].contiguous(), Td[perm].contiguous()
    losses = []
    nb = max(1, Xd.shape[0] // batch)
    for ep in range(epochs):
        tot = 0.0
        for b in range(nb):
            xs, ts = Xd[b * batch:(b + 1) * batch], Td[b * batch:(b + 1) * batch]
            want = (b % 50 == 0) or b == nb - 1
            l = tr.step(xs, ts, lr, want_loss=want)
            if want:
                tot = l if tot == 0.0 else 0.5 * (tot + l)
        losses.append(tot)
    p = tr.params()
    tr.close()
    return p, losses
