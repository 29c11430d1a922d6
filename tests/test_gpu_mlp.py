"""Learned warm start on the GPU against the FP64 oracle.

- Inference: the fused BF16 tensor-core forward vs the oracle's FP64 forward on
  the same features (relative error of a BF16 network, <= 3e-2 of the output scale).
- Gradients: the trainer's backward vs the oracle's backpropagation, per tensor
  cosine >= 0.999 and relative L2 <= 2e-2 (BF16 operands, FP32 accumulation).
- Training decreases the loss on impulses logged from the plain solver.
- Physics with the learned warm start, iterated to the 1e-6 residual, agrees
  with the oracle in learned mode from an identical state.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from parity import identical_start, step_both_and_compare

pytestmark = pytest.mark.gpu

OFFS = [("W1", 0, 4096), ("b1", 4096, 4224), ("W2", 4224, 20608), ("b2", 20608, 20736), ("W3", 20736, 37120),
        ("b3", 37120, 37248), ("W4", 37248, 37632), ("b4", 37632, 37635)]


def _logged(n_envs=64, steps=6, warm=30):
    from paper_2106_14405_gb300.learn import collect
    p = sg.params_for(4)
    b = sg.make_batch(2, n_envs)
    return collect(b, p, steps, warm_steps=warm)


def test_inference_matches_fp64_forward():
    from paper_2106_14405_gb300.learn import Trainer
    X, _ = _logged(32, 2)
    assert len(X) > 100
    P = sg.mlp_init(1)
    P[4096:4224] = np.random.default_rng(2).normal(0, 0.1, 128)
    tr = Trainer(P, len(X))
    Y = tr.forward(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()
    ref = O.mlp_forward(P, X.astype(np.float64))
    scale = np.abs(ref).max()
    assert np.abs(Y - ref).max() <= 3e-2 * scale, (np.abs(Y - ref).max(), scale)


def test_gradients_match_oracle_backprop():
    from paper_2106_14405_gb300.learn import Trainer
    rng = np.random.default_rng(3)
    n = 512
    X = rng.normal(size=(n, 32))
    T = rng.normal(size=(n, 3))
    P = sg.mlp_init(4)
    P[4096:4224] = rng.normal(0, 0.1, 128)
    tr = Trainer(P, n)
    loss, g = tr.loss_grad(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    ref_loss, ref = O.mlp_loss_grad(P, X, T)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    for name, a, b in OFFS:
        x, y = g[a:b], ref[a:b]
        cos = x @ y / (np.linalg.norm(x) * np.linalg.norm(y))
        rel = np.linalg.norm(x - y) / np.linalg.norm(y)
        assert cos >= 0.999 and rel <= 2e-2, (name, cos, rel)


def test_training_reduces_loss():
    from paper_2106_14405_gb300.learn import train
    X, T = _logged(128, 8)
    P0 = sg.mlp_init(0)
    _, losses = train(X, T, P0, epochs=6, batch=1024, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0], losses


def test_learned_mode_physics_parity_at_residual():
    b = sg.make_batch(4, 32)
    p = sg.params_for(4)
    p.warm_mode = 2
    P = sg.mlp_init(5) * 0.1
    from paper_2106_14405_gb300 import Sim
    sim = Sim(b, p)
    sim.set_mlp(P)
    orc = O.Oracle(b, p)
    orc.set_mlp(P)
    sim.step(30)
    err, flips, _, _ = step_both_and_compare(b, sim, orc)
    assert flips.mean() <= 0.1
    for k, v in err.items():
        tol = 1e-3 if k in ("obj_omega", "joint_qd_revolute") else 1e-4
        assert v <= tol, (k, v)
