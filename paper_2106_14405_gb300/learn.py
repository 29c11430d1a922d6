"""Learned PGS warm start: dataset logging and training through the C ABI.

The network predicts, per contact, the correction from the prior-frame impulses
to the converged impulses (normal, two friction), divided by m_eff,n |g| dt,
from 32 contact features (which include the prior-frame impulses); the
deployed warm start (sim_set_mlp, warm_mode 2) uses it for contacts that have
no prior-frame match and keeps the prior impulse for the others, so training
uses the unmatched contacts (feature 26 = 0).  Every computation runs in the
library's kernels: logging in the
simulator step, forward/backward/Adam in the trainer; this module only moves
arguments and orders the minibatches.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N
from .engine import Sim

NPARAM = 128 * 32 + 128 + 2 * (128 * 128 + 128) + 3 * 128 + 3


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


def collect(batch, params, steps: int, warm_steps: int = 0, cap_per_step: int = 1 << 20):
    """Run the plain solver (prior-frame warm start) to the params' residual target and
    return the logged (features, normalised impulse corrections) of every contact of
    every step as host arrays."""
    sim = Sim(batch, params, use_graph=False, log_features=True)
    if warm_steps:
        sim.step(warm_steps)
    feats, lams = [], []
    for _ in range(steps):
        sim.step(1)
        f, l, n = sim.log_contacts(cap_per_step)
        st = sim.stats()
        sim.sync()
        # keep contacts of environments whose solve reached the residual target this step
        keep = np.repeat((st["status"] & 4) == 0, st["n_contacts"])[:len(f)]
        feats.append(f.cpu().numpy()[keep])
        lams.append(l.cpu().numpy()[keep])
    sim.close()
    return np.concatenate(feats), np.concatenate(lams)


def train(X: np.ndarray, T: np.ndarray, init_params, epochs: int = 3, batch: int = 4096, lr: float = 1e-3,
          seed: int = 0, clip: float = 10.0, new_only: bool = True):
    """Adam on minibatches of a fixed seeded permutation of the data (the contacts without a
    prior-frame match when new_only), targets clipped to [-clip, clip] (the heavy tail of
    impulse corrections otherwise dominates the squared error); returns (params for raw
    features, list of per-epoch mean losses)."""
    T = np.clip(T, -clip, clip)
    if new_only:
        sel = X[:, 26] == 0
        X, T = X[sel], T[sel]
    mean = X.mean(0)
    std = X.std(0)
    std[std < 1e-6] = 1.0
    tr = Trainer(init_params, batch, mean, std)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(X))
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm], np.float32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T[perm], np.float32)).cuda()
    losses = []
    nb = max(1, len(X) // batch)
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
