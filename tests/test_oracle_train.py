"""Pins of the oracle's training loss and gradient (Sec. 3.3: Eq. 4 summed over every tail with
the L1 SDF loss of Eq. 8) and of its Adam step (Sec. 4.1).

* A float64 torch restatement of the loss, differentiated by torch's autograd, gives the same
  gradient for every parameter (SIREN with linear and multiplicative tails, FINER, ReLU on
  Fourier features whose matrix is not trained).
* Central differences of the oracle's own loss along random parameter directions match the
  gradient (points kept a margin away from the kinks y_i = y_gt of the L1 loss).
* The hand-built sphere model, whose cumulative outputs are y_1 = -r^2, y_2 = x^2 - r^2,
  y_3 = x^2 + y^2 - r^2, y_4 = |x|^2 - r^2, has closed-form derivatives: the tail-1 bias
  enters every y_i, so dL/dc_1 = (1/n) sum_x sum_i sign(y_i - y_gt); the first factor bias of
  tail 2 multiplies x, so dL/dc_2 = (1/n) sum_x x G_2 with G_2 = sum_{i>=2} sign(y_i - y_gt);
  the bias of the x+ unit of layer 1 reaches tail 2 through (x+ - x-)^2, so dL/db1[0] =
  (1/n) sum_x 2 x G_2 [x > 0].
* The Adam step equals torch.optim.Adam's over several steps.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
import synth


def unflatten(model, flat):
    """A copy of `model` with its parameter block replaced by `flat` (model.flat() order)."""
    flat = np.asarray(flat)
    L, W, D, m = model.n_layers, model.width, model.in_dim, model.n_freq
    o = 0
    out = {}
    if model.encoder == synth.ENC_FOURIER:
        out["enc_B"] = flat[o:o + m * 3].reshape(m, 3); o += m * 3
    for name, shape in (("W1", (W, D)), ("b1", (W,)), ("Wh", (L - 1, W, W)), ("bh", (L - 1, W)),
                        ("tail_w", (L, 2, W)), ("tail_b", (L, 2))):
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    assert o == flat.size
    return out


def torch_loss_grad(model, pts, gt):
    """Eq. 4 / Eq. 8 restated with float64 torch tensors; the gradient by autograd, flattened in
    the parameter-block order (the Fourier matrix gets zeros: it is not trained)."""
    dt = torch.float64
    x = torch.tensor(np.asarray(pts, np.float64))
    target = torch.tensor(np.asarray(gt, np.float64))
    P = {k: torch.tensor(getattr(model, k).astype(np.float64), requires_grad=True)
         for k in ("W1", "b1", "Wh", "bh", "tail_w", "tail_b")}
    if model.encoder == synth.ENC_FOURIER:
        B = torch.tensor(model.enc_B.astype(np.float64))
        s = 2 * math.pi * (x @ B.T)
        h = torch.cat([torch.sin(s), torch.cos(s)], dim=1)
    else:
        h = x
    w0 = model.omega0
    y = torch.zeros(x.shape[0], dtype=dt)
    loss = torch.zeros((), dtype=dt)
    for l in range(1, model.n_layers + 1):
        Wl = P["W1"] if l == 1 else P["Wh"][l - 2]
        bl = P["b1"] if l == 1 else P["bh"][l - 2]
        u = h @ Wl.T + bl
        if model.activation == synth.ACT_RELU:
            h = torch.relu(u)
        elif model.activation == synth.ACT_FINER:
            h = torch.sin(w0 * (u.abs() + 1) * u)
        else:
            h = torch.sin(w0 * u)
        t = h @ P["tail_w"][l - 1, 0] + P["tail_b"][l - 1, 0]
        if model.tail_kind == synth.TAIL_MULT and l >= 2:
            t = t * (h @ P["tail_w"][l - 1, 1] + P["tail_b"][l - 1, 1])
        y = y + t
        loss = loss + (y - target).abs().mean()
    loss.backward()
    parts = []
    if model.encoder == synth.ENC_FOURIER:
        parts.append(np.zeros(model.enc_B.size))
    for k in ("W1", "b1", "Wh", "bh", "tail_w", "tail_b"):
        parts.append(P[k].grad.numpy().ravel())
    return float(loss.detach()), np.concatenate(parts)


def scene_targets(pts):
    return synth.scene_sdf(np.asarray(pts, np.float64)).astype(np.float32)


MODELS = {
    "siren": lambda: synth.siren_tmlp(4, 24, seed=31),
    "siren_mult": lambda: synth.siren_tmlp(4, 24, seed=32, tail_kind=synth.TAIL_MULT),
    "finer": lambda: synth.finer_tmlp(3, 20, seed=33),
    "relu_ff": lambda: synth.relu_ff_tmlp(3, 24, n_freq=12, sigma=3.0, seed=34),
}


@pytest.mark.parametrize("kind", sorted(MODELS))
def test_train_grad_matches_torch_autograd(kind):
    model = MODELS[kind]()
    pts = synth.uniform_points(400, seed=35)
    gt = scene_targets(pts)
    loss, g = oracle.train_grad(model, pts, gt)
    loss_t, g_t = torch_loss_grad(model, pts, gt)
    assert abs(loss - loss_t) <= 1e-12 * max(1.0, abs(loss_t))
    scale = max(1e-3, float(np.abs(g_t).max()))
    assert np.abs(g - g_t).max() <= 1e-11 * scale, np.abs(g - g_t).max()
    assert np.abs(g_t).max() > 0


@pytest.mark.parametrize("kind", ["siren", "siren_mult", "finer"])
def test_train_grad_central_differences(kind):
    model = MODELS[kind]()
    pts = synth.uniform_points(600, seed=36)
    gt = scene_targets(pts)
    _, ys = oracle.evaluate(model, pts, model.n_layers, all_tails=True)
    keep = np.abs(ys - gt.astype(np.float64)[:, None]).min(axis=1) > 1e-3  # away from the L1 kinks
    pts, gt = pts[keep], gt[keep]
    _, g = oracle.train_grad(model, pts, gt)
    base = model.flat().astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(37))
    for _ in range(3):
        v = rng.standard_normal(base.size) * np.maximum(np.abs(base), 1e-3)
        plus = (base + 1e-5 * v).astype(np.float32)
        minus = (base - 1e-5 * v).astype(np.float32)
        step = plus.astype(np.float64) - minus.astype(np.float64)  # the perturbation float32 represents
        lp, _ = oracle.train_grad(dataclasses.replace(model, **unflatten(model, plus)), pts, gt)
        lm, _ = oracle.train_grad(dataclasses.replace(model, **unflatten(model, minus)), pts, gt)
        fd = lp - lm
        an = float(g @ step)
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-12, (fd, an)


def test_train_grad_closed_form_sphere():
    r = 0.6
    model = synth.relu_sphere_tmlp(r, width=8)
    pts = synth.uniform_points(3000, seed=38)
    p = pts.astype(np.float64)
    gt = (np.linalg.norm(p, axis=1) - r).astype(np.float32)
    g64 = gt.astype(np.float64)
    r2 = float(np.float32(-r * r))  # the tail-1 bias as stored (float32)
    ys = [r2 + 0 * p[:, 0], r2 + p[:, 0] ** 2, r2 + p[:, 0] ** 2 + p[:, 1] ** 2, r2 + (p ** 2).sum(1)]
    sg = [np.sign(y - g64) for y in ys]
    n = len(pts)
    G2 = sg[1] + sg[2] + sg[3]
    _, g = oracle.train_grad(model, pts, gt)
    parts = unflatten(model, g)
    assert abs(parts["tail_b"][0, 0] - sum(s.sum() for s in sg) / n) <= 1e-12
    assert abs(parts["tail_b"][1, 0] - (p[:, 0] * G2).sum() / n) <= 1e-12
    assert abs(parts["b1"][0] - (2 * p[:, 0] * G2 * (p[:, 0] > 0)).sum() / n) <= 1e-12
    loss, _ = oracle.train_grad(model, pts, gt)
    assert abs(loss - sum(np.abs(y - g64).mean() for y in ys)) <= 1e-12


def test_adam_matches_torch():
    rng = np.random.Generator(np.random.PCG64(39))
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * 10.0 ** rng.uniform(-6, 0) for _ in range(4)]
    w = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-4, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, gr in enumerate(grads, start=1):
        w.grad = torch.tensor(gr)
        opt.step()
        p, m, v = oracle.adam_step(p, gr, m, v, t)
        assert np.abs(p - w.detach().numpy()).max() <= 1e-15
