"""T-MLP training steps (Sec. 3.3: Eq. 4 with the L1 SDF loss of Eq. 8; Adam of Sec. 4.1) through
the C-ABI (sand_trainer_*, sand_train_step) against the FP64 oracle (oracle.train_grad,
oracle.adam_step).

The tensor-core products are float32-class (split fp16 operands, float32 accumulation), so the
loss is held to a relative 1e-5 and the gradient of every parameter group (W_1, b_1, the hidden
W_l and b_l, the tail weights and the tail biases) to 1e-5 omega0 max|g| of its group: one
derivative of sin(omega0 z) multiplies the sensitivity to rounding by omega0, as for the input
gradient.  The L1 loss has kinks where y_i = y_gt, at which the two sides may take different
signs, so the batches keep points whose min_i |y_i - y_gt| exceeds 1e-3 (the oracle decides).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def groups(model, flat):
    L, W, D = model.n_layers, model.width, model.in_dim
    o = 0
    out = {}
    for name, k in (("W1", W * D), ("b1", W), ("Wh", (L - 1) * W * W), ("bh", (L - 1) * W), ("tail_w", L * 2 * W),
                    ("tail_b", L * 2)):
        out[name] = np.asarray(flat[o:o + k], np.float64)
        o += k
    return out


def batch(model, n, seed, margin=1e-3):
    g = np.random.Generator(np.random.PCG64(seed))
    pts = g.uniform(-1, 1, (3 * n + 64, 3)).astype(np.float32)
    gt = synth.scene_sdf(pts.astype(np.float64)).astype(np.float32)
    _, ys = oracle.evaluate(model, pts, model.n_layers, all_tails=True)
    keep = np.abs(ys - gt.astype(np.float64)[:, None]).min(axis=1) > margin
    pts, gt = pts[keep][:n], gt[keep][:n]
    assert len(pts) == n
    return pts, gt


def load(model):
    from paper_2604_25936_gb300 import Model
    return Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)


def check_step(model, pts, gt, what):
    from paper_2604_25936_gb300.binding import Trainer
    m = load(model)
    tr = Trainer(m, max_points=max(len(pts), 1))
    grad = torch.empty(tr.n_params, dtype=torch.float32, device="cuda")
    loss, _ = tr.step(torch.from_numpy(pts).cuda(), torch.from_numpy(gt).cuda(), update=False, grad=grad)
    torch.cuda.synchronize()
    tr.status()
    loss_ref, g_ref = oracle.train_grad(model, pts, gt)
    lv = float(loss.item())
    assert abs(lv - loss_ref) <= 1e-5 * abs(loss_ref), (what, lv, loss_ref)
    gg = groups(model, grad.double().cpu().numpy())
    gr = groups(model, g_ref)
    w0 = model.omega0 if model.activation != synth.ACT_RELU else 30.0
    worst = {}
    for name in gg:
        scale = float(np.abs(gr[name]).max())
        err = float(np.abs(gg[name] - gr[name]).max())
        worst[name] = err / max(scale, 1e-30)
        if scale == 0.0:
            assert err == 0.0, (what, name, err)
            continue
        assert err <= 1e-5 * w0 * scale, (what, name, err, scale)
    print("train %s: loss %.6g (oracle %.6g); max |dg| / max |g| per group %s"
          % (what, lv, loss_ref, {k: "%.2e" % v for k, v in worst.items()}))
    return m, tr, grad


@pytest.mark.parametrize("kind,width,n", [("siren", 64, 3001), ("siren", 128, 129), ("siren", 256, 128),
                                          ("siren_mult", 256, 4097), ("finer", 64, 1000), ("relu", 64, 2000)])
def test_train_step_gradient_matches_oracle(kind, width, n):
    if kind == "siren":
        model = synth.siren_tmlp(4, width, seed=41)
    elif kind == "siren_mult":
        model = synth.siren_tmlp(8, width, seed=42, tail_kind=synth.TAIL_MULT)
    elif kind == "finer":
        model = synth.finer_tmlp(4, width, seed=43)
    else:
        model = synth.relu_sphere_tmlp(0.6, width=width)
    pts, gt = batch(model, n, seed=n + width)
    m, tr, _ = check_step(model, pts, gt, "%s/%d/n=%d" % (kind, width, n))
    tr.close()
    m.free()


def test_train_step_one_point():
    model = synth.siren_tmlp(3, 64, seed=44)
    pts, gt = batch(model, 1, seed=45)
    m, tr, _ = check_step(model, pts, gt, "one point")
    tr.close()
    m.free()


def test_train_step_benchmark_model():
    """The benchmark's 8 x 256 SIREN (linear tails) on 20,000 points."""
    model = synth.siren_tmlp(8, 256, seed=1)
    pts, gt = batch(model, 20000, seed=46)
    m, tr, _ = check_step(model, pts, gt, "8x256/n=20000")
    tr.close()
    m.free()


def test_adam_update_and_commit():
    """The update applied by a step is the Adam step of the gradient the same step produced (the
    oracle's Adam, float64, on that float32 gradient); after a commit the model answers queries
    with the trained parameters."""
    from paper_2604_25936_gb300.binding import Trainer
    model = synth.siren_tmlp(4, 64, seed=47)
    pts, gt = batch(model, 2000, seed=48)
    m = load(model)
    tr = Trainer(m, max_points=4096, lr=1e-3)
    x, t = torch.from_numpy(pts).cuda(), torch.from_numpy(gt).cuda()
    p0 = tr.params().astype(np.float64)
    mom, vel = np.zeros_like(p0), np.zeros_like(p0)
    p_ref = p0
    for step in range(1, 4):
        grad = torch.empty(tr.n_params, dtype=torch.float32, device="cuda")
        tr.step(x, t, update=True, grad=grad)
        torch.cuda.synchronize()
        p_ref, mom, vel = oracle.adam_step(p_ref, grad.double().cpu().numpy(), mom, vel, step, lr=1e-3)
        p = tr.params().astype(np.float64)
        assert np.abs(p - p_ref).max() <= 1e-6 * max(1.0, float(np.abs(p_ref).max())), step
    tr.commit()
    trained = dataclasses.replace(model, **{k: v.astype(np.float32).reshape(getattr(model, k).shape)
                                            for k, v in groups(model, tr.params()).items()})
    q = synth.uniform_points(3000, seed=49)
    y = m.query(torch.from_numpy(q).cuda(), precision="fp32", full_depth=True).double().cpu().numpy()
    assert np.abs(y - oracle.full_depth(trained, q)).max() <= 1e-5
    tr.close()
    m.free()


def test_training_lowers_the_loss():
    """200 steps of Adam (learning rate 1e-3) on one batch of scene SDF targets lower the loss of
    Eq. 4 / Eq. 8 by a fifth at least; the first step's loss is the oracle's."""
    from paper_2604_25936_gb300.binding import Trainer
    model = synth.siren_tmlp(4, 128, seed=50)
    pts, gt = batch(model, 8192, seed=51, margin=0.0)
    m = load(model)
    tr = Trainer(m, max_points=8192, lr=1e-3)
    x, t = torch.from_numpy(pts).cuda(), torch.from_numpy(gt).cuda()
    losses = []
    for _ in range(200):
        loss, _ = tr.step(x, t)
        losses.append(loss)
    torch.cuda.synchronize()
    tr.status()
    first, last = float(losses[0].item()), float(losses[-1].item())
    l0, _ = oracle.train_grad(model, pts, gt)
    assert abs(first - l0) <= 1e-5 * l0
    assert last < 0.8 * first, (first, last)
    tr.close()
    m.free()


def test_trainer_refuses_what_it_does_not_take():
    from paper_2604_25936_gb300 import SandError
    from paper_2604_25936_gb300.binding import Trainer
    ff = synth.relu_ff_tmlp(3, 64, n_freq=32, sigma=4.0, seed=52)
    m = load(ff)
    with pytest.raises(SandError, match="EUNSUPPORTED"):
        Trainer(m)
    m.free()
    model = synth.siren_tmlp(3, 64, seed=53)
    m = load(model)
    tr = Trainer(m, max_points=256)
    x = torch.zeros((300, 3), device="cuda")
    with pytest.raises(SandError, match="EINVAL"):
        tr.step(x, torch.zeros(300, device="cuda"))
    tr.close()
    m.free()
