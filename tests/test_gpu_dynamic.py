"""Octree-free dynamic exit (Table 6) through sand_query_sdf_dynamic, against the FP64 oracle.

A point stops at the first layer whose tail |t_i| < r.  As with every decision taken on
floating-point values, the GPU (float32-class) and the oracle (float64) may part only
where |t_i| is within the output tolerance of r; per point the test allows the range of
exit layers such close calls permit and checks the value at the GPU's exit layer.
Tiles whose rows have all stopped skip their remaining layers: a point set arranged so
that whole tiles stop early, between tiles that run to the end, checks that the skipped
weight stages and the accumulator hand-over stay in step.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def load(model):
    from paper_2604_25936_gb300 import Model
    return Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)


def exit_range(ys, r, tol=TOL):
    t = np.diff(np.concatenate([np.zeros((ys.shape[0], 1)), ys], axis=1), axis=1)
    maybe = np.abs(t) < r + 2 * tol
    sure = np.abs(t) < r - 2 * tol
    maybe[:, -1] = True
    sure[:, -1] = True
    return np.argmax(maybe, axis=1) + 1, np.argmax(sure, axis=1) + 1


def check(m, model, pts, r, prec="fp32"):
    y, el = m.query_dynamic(torch.from_numpy(pts).cuda(), r=r, precision=prec)
    y = y.double().cpu().numpy()
    el = el.cpu().numpy().astype(np.int64)
    y_ref, d_ref, ys = oracle.dynamic_exit(model, pts, r)
    lo, hi = exit_range(ys, r)
    assert ((el >= lo) & (el <= hi)).all(), "exit layer outside the range the tolerance allows"
    fixed = lo == hi
    np.testing.assert_array_equal(el[fixed], d_ref[fixed])
    err = np.abs(y - ys[np.arange(len(el)), el - 1]).max()
    assert err <= TOL * max(1.0, float(np.abs(ys).max())), err
    return el, d_ref


@pytest.mark.parametrize("r", [1.5e-4, 0.05])
def test_dynamic_siren(r):
    model = synth.siren_tmlp(8, 256, seed=1)
    m = load(model)
    el, d_ref = check(m, model, synth.uniform_points(20001, seed=43), r)
    if r > 0.01:
        assert len(np.unique(el)) > 3  # rows stop at many different layers
    m.free()


def test_dynamic_sphere_tiles_skip():
    """Closed-form model (tails -R^2, x^2, y^2, z^2), r = 0.01: tiles of points with |x| < 0.05
    all stop at layer 2 (whole-tile skip), tiles with every coordinate >= 0.3 run to layer 4;
    640 tiles, so every CTA meets both kinds one after the other."""
    model = synth.relu_sphere_tmlp(0.6, width=64)
    m = load(model)
    g = np.random.Generator(np.random.PCG64(5))
    tiles = []
    for k in range(640):  # several tiles per CTA (one CTA per SM), in mixed order
        if k % 3 == 2:
            p = g.uniform(0.3, 0.9, (128, 3))
        else:
            p = np.stack([g.uniform(-0.05, 0.05, 128), g.uniform(0.3, 0.9, 128), g.uniform(0.3, 0.9, 128)], 1)
        tiles.append(p)
    pts = np.concatenate(tiles + [g.uniform(-1, 1, (77, 3))]).astype(np.float32)  # and a ragged tail
    el, d_ref = check(m, model, pts, 1e-2)
    assert (el[:128] == 2).all() and (el[2 * 128:3 * 128] == 4).all()
    # the same points again, one at a time through the full-depth path agree at layer L
    full = m.query(torch.from_numpy(pts).cuda(), full_depth=True, precision="fp32").double().cpu().numpy()
    _, _, ys = oracle.dynamic_exit(model, pts, 1e-2)
    assert np.abs(full - ys[:, -1]).max() <= TOL
    m.free()


@pytest.mark.parametrize("kind", ["siren", "sphere"])
def test_dynamic_every_tile_stops_at_layer_1(kind):
    """r above every |t_1|: every row stops at layer 1, so every tile of every CTA is skipped one
    after the other, with no MMA between the skips (layer 1 of the SIREN's raw coordinates runs on
    the CUDA cores; the sphere's multiplicative tails keep it as one MMA).  The kernel must hand
    each skip to the MMA thread in turn: all exit layers 1, values t_1, no timeout."""
    if kind == "siren":
        model = synth.siren_tmlp(8, 256, seed=1)
    else:
        model = synth.relu_sphere_tmlp(0.6, width=64)
    m = load(model)
    pts = synth.uniform_points(300001, seed=47)
    _, _, ys = oracle.dynamic_exit(model, pts[:20000], 1e9)
    r = float(1.5 * np.abs(ys[:, 0]).max() + 0.1)
    y, el = m.query_dynamic(torch.from_numpy(pts).cuda(), r=r)
    st = m.stats()  # the model's own workspace; raises SandError (ETIMEOUT) if a wait ran out
    assert not (st["flags"] & 2), "a device-side wait timed out"
    assert (el.cpu().numpy() == 1).all()
    idx = synth.sample_indices(len(pts), 20000, seed=3)
    y_ref, d_ref, _ = oracle.dynamic_exit(model, pts[idx], r)
    assert (d_ref == 1).all()
    assert np.abs(y.double().cpu().numpy()[idx] - y_ref).max() <= TOL
    m.free()


def test_dynamic_errors():
    from paper_2604_25936_gb300 import SandError
    model = synth.siren_tmlp(4, 64, seed=0)
    m = load(model)
    x = torch.zeros((10, 3), device="cuda")
    with pytest.raises(SandError, match="EINVAL"):
        m.query_dynamic(x, r=0.0)
    with pytest.raises(SandError, match="EUNSUPPORTED"):
        m.query_dynamic(x, precision="fp32_simt")
    m.free()
