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


@pytest.mark.parametrize("use_graph,out_bias", [(False, 0.1), (True, 0.1), (True, 12.0)])
def test_step_inference_matches_fp64_forward(use_graph, out_bias):
    """The in-step inference (tensor-core forward in 128-row tiles over the
    contacts the network serves, which the row kernel lists) against the oracle's
    FP64 forward on the same logged features."""
    from paper_2106_14405_gb300 import Sim
    b = sg.make_batch(2, 1024)
    p = sg.params_for(2)
    p.warm_mode = 2
    P = sg.mlp_init(7)
    rng = np.random.default_rng(7)
    for a, z in ((4096, 4224), (20608, 20736), (37120, 37248)):
        P[a:z] = rng.normal(0, 0.1, z - a)  # non-zero biases
    P[37632:37635] = rng.normal(0, out_bias, 3)  # with 12, outputs past the +-10 limit
    sim = Sim(b, p, use_graph=use_graph, log_features=True)
    sim.set_mlp(P)
    sim.step(40)
    sim.step(1)
    X, _, n = sim.log_contacts(1 << 16)
    Y, n2 = sim.log_predictions(1 << 16)
    assert n == n2 and n > 1000
    Xh = X.cpu().numpy().astype(np.float64)
    # the rows the network ran on: no prior-frame match, or a relative velocity above
    # 4 |g| dt (decided in FP32 on the device: rows within rounding of the gate left out)
    speed = np.linalg.norm(Xh[:, 9:12], axis=1)
    gate = 4 * 9.81 * p.dt
    new = (Xh[:, 26] == 0) | (speed > gate * (1 + 1e-5))
    assert new.sum() > 128  # more than one tile
    # the batch statistics count the rows the network served (the log leaves out rows
    # without a finite target, which the network may still have served)
    tot = sim.totals()
    near = (Xh[:, 26] == 0) | (speed > gate * (1 - 1e-5))
    assert new.sum() <= tot["n_net_rows"] <= near.sum() + (tot["n_contacts"] - n)
    ref = np.clip(O.mlp_forward(P, Xh[new]), -10, 10)  # the in-step output limit
    Yh = Y.cpu().numpy()[new]
    scale = np.abs(ref).max()
    assert np.abs(Yh - ref).max() <= 3e-2 * scale, (np.abs(Yh - ref).max(), scale)
    assert sim.sync()[1] & 16 == 0  # no device wait gave up


@pytest.mark.parametrize("out", [(4.0, -3.0, 2.5), (25.0, -30.0, 3.0)])
def test_learned_warm_start_application_parity_fixed_sweeps(out):
    """The step with the learned warm start at the workload's fixed sweep count, where
    the start decides the result: a network with a constant output (W4 = 0, b4 = out)
    gives the same prediction on both sides exactly, so the GPU's use of it (scale,
    output limit of +-10, projection onto the friction pyramid) must match the oracle."""
    from paper_2106_14405_gb300 import Sim
    b = sg.make_batch(2, 256)
    p = sg.params_for(2)
    P = np.zeros(len(sg.mlp_init(0)))
    P[37632:37635] = out
    warm = Sim(b, p)
    warm.step(30)
    s0 = warm.get_state()
    s0["cache_count"][:] = 0  # every contact is new: the network serves them all
    q = sg.params_for(2)
    q.warm_mode = 2
    sim = Sim(b, q)
    sim.set_mlp(P)
    sim.set_state(s0)
    orc = O.Oracle(b, q)
    orc.set_mlp(P)
    err, flips, _, _ = step_both_and_compare(b, sim, orc)
    assert flips.mean() <= 0.1
    for k, v in err.items():
        tol = 1e-3 if k in ("obj_omega", "joint_qd_revolute") else 1e-4
        assert v <= tol, (k, v)
    assert sim.sync()[1] & 16 == 0


def test_trainer_rejects_unaligned_features():
    """The forward reads each row's features as 16-byte vectors: an X that is not
    16-byte aligned is refused (SIM_ERR_INVALID_ARG) before any launch; a row slice
    of an allocation is aligned and runs."""
    from paper_2106_14405_gb300 import SimError
    from paper_2106_14405_gb300.learn import Trainer
    P = sg.mlp_init(1)
    tr = Trainer(P, 256)
    X = torch.randn(257 * 32 + 1, device="cuda")
    T = torch.zeros(256, 3, device="cuda")
    bad = X[1:1 + 256 * 32].view(256, 32)  # 4 bytes past the allocation's start
    for call in (lambda: tr.forward(bad), lambda: tr.loss_grad(bad, T), lambda: tr.step(bad, T, 1e-3)):
        with pytest.raises(SimError) as ei:
            call()
        assert ei.value.code == 1
    rows = X[:257 * 32].view(257, 32)[1:]  # a row slice: 128 bytes in
    ref = tr.forward(rows.contiguous().clone())
    assert torch.equal(tr.forward(rows), ref)


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


def test_adam_step_matches_numpy_adam_elementwise():
    """Two trainer steps against Adam written out from Kingma & Ba (2015) in NumPy on
    the trainer's own gradients: m_t = b1 m + (1 - b1) g, v_t = b2 v + (1 - b2) g^2,
    p -= lr (m_t / (1 - b1^t)) / (sqrt(v_t / (1 - b2^t)) + eps), b1 0.9, b2 0.999,
    eps 1e-8 outside the square root.  Each step's gradient is taken at the trainer's
    parameters before the step (the same deterministic kernels the step runs)."""
    from paper_2106_14405_gb300.learn import Trainer
    rng = np.random.default_rng(21)
    n = 384
    X = torch.from_numpy(rng.normal(size=(n, 32)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).cuda()
    P = sg.mlp_init(6).astype(np.float32)
    tr = Trainer(P, n)
    lr, b1, b2, eps = 3e-3, 0.9, 0.999, 1e-8
    p = P.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in (1, 2):
        _, g = tr.loss_grad(X, T)
        g = g.cpu().numpy().astype(np.float64)
        tr.step(X, T, lr)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        got = tr.params().astype(np.float64)
        # FP32 arithmetic on the device: the update (~lr) to a few FP32 ulps of the parameter
        tol = 1e-6 * np.maximum(1.0, np.abs(p)) + 1e-4 * lr
        bad = np.abs(got - p) > tol
        assert not bad.any(), (t, int(bad.sum()), float(np.abs(got - p).max()))
        p = got  # continue from the device's FP32 parameters


def test_training_reduces_loss():
    from paper_2106_14405_gb300.learn import train
    X, T = _logged(128, 8)
    P0 = sg.mlp_init(0)
    _, losses = train(X, T, P0, epochs=6, batch=1024, lr=1e-3)
    assert losses[-1] < 0.6 * losses[0], losses


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


def test_trained_network_gain_over_prior_frame():
    """What the learned warm start gains over the method without it (the prior-frame
    warm start, which starts new contacts at zero and keeps every matched contact's
    last impulse): a lower held-out error on the impulses of the contacts the network
    serves, and fewer PGS sweeps to the 1e-6 residual on held-out scenes, over the
    env-steps that converge in every mode."""
    from paper_2106_14405_gb300 import Sim
    from paper_2106_14405_gb300.learn import Trainer, collect, train
    p = sg.params_for(4)
    X, T = collect(sg.make_batch(2, 4096, seed_offset=2_000_000), p, 40, warm_steps=20, device=True)
    params, losses = train(X, T, sg.mlp_init(0), epochs=6, batch=4096, lr=1e-3)
    Xh, Th = collect(sg.make_batch(4, 256, seed_offset=500_000), p, 6, warm_steps=30)
    served = (Xh[:, 26] == 0) | (np.linalg.norm(Xh[:, 9:12], axis=1) > 4 * 9.81 * p.dt)
    Xh, Th = Xh[served], np.clip(Th[served], -10, 10)
    tr = Trainer(params, len(Xh))
    Yh = tr.forward(torch.from_numpy(Xh.astype(np.float32)).cuda()).cpu().numpy()
    mse_learned = float(((Yh - Th) ** 2).mean())
    mse_prior = float((Th ** 2).mean())
    held = sg.make_batch(4, 2048, seed_offset=600_000)
    base = Sim(held, p)
    base.step(30)
    start = base.get_state()
    its = {}
    for name, mode in (("cold", 0), ("prior", 1), ("learned", 2)):
        q = sg.params_for(4)
        q.warm_mode = mode
        sim = Sim(held, q)
        if mode == 2:
            sim.set_mlp(params)
        sim.set_state(start)
        rows = []
        for _ in range(8):
            sim.step(1)
            st = sim.stats()
            rows.append(np.where((st["n_rows"] > 0) & ((st["status"] & 4) == 0), st["iters"], -1))
            sim.sync()
        its[name] = np.stack(rows)
    ok = np.ones_like(its["cold"], bool)
    for v in its.values():
        ok &= v >= 0
    mean = {k: float(v[ok].mean()) for k, v in its.items()}
    print("held-out correction MSE learned %.3f vs prior-frame %.3f; mean sweeps to 1e-6 %s; training loss %s"
          % (mse_learned, mse_prior, mean, losses))
    assert mse_learned < 0.5 * mse_prior
    assert mean["learned"] < mean["prior"], mean
