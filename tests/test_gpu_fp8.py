"""FP8 (e4m3) hidden-layer products on the tensor cores, against the FP64 oracle.

e4m3 keeps 3 mantissa bits (unit roundoff 2^-4), so the FP8 mode is an
approximation whose error is reported, not bounded by the float32 tolerance.
The bounds come from tests/quantised_emulation.py, which rounds the same
operands the same way (per-layer power-of-two weight scale, unscaled sine
activations) and does everything else in float64: its error against the
oracle at full depth on 20,000 uniform points (PCG64 seed 17), per model
(8 x 256: 2.3e-2 max, 5.6e-3 RMS; 8 x 336: 2.9e-2 / 5.7e-3; 4 x 64:
1.3e-2 / 3.0e-3).  A test allows 3x that maximum and 2x that RMS; full depth
bounds the SAND queries too, whose rows stop earlier.  Points that exit at
layer 1 never touch the tensor cores (layer 1 is float32), so they keep the
float32 tolerance, and exit layers stay bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import quantised_emulation as qe
import synth

pytestmark = pytest.mark.gpu


def fp8_bounds(model, grad=False):
    """(max, RMS) bounds: 3x and 2x the emulated FP8 error at full depth."""
    emax, erms = qe.full_depth_error(model, "fp8", grad=grad)
    return 3.0 * emax, 2.0 * erms


def load(model, tree=None):
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    if tree is not None:
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def check_fp8(y_gpu, y_ref, d_ref, what, bounds):
    max_tol, rms_tol = bounds
    y = y_gpu.double().cpu().numpy() if isinstance(y_gpu, torch.Tensor) else np.asarray(y_gpu, np.float64)
    assert np.isfinite(y).all(), what + ": non-finite output"
    err = np.abs(y - y_ref)
    if d_ref is not None:
        one = d_ref == 1
        if one.any():
            assert err[one].max() <= 1e-5, "%s: exit-layer-1 rows |err| %.3g" % (what, err[one].max())
        zero = d_ref == 0
        if zero.any():
            assert err[zero].max() == 0 or err[zero].max() <= 1e-7, what + ": far leaves changed"
    rms = float(np.sqrt((err ** 2).mean())) if err.size else 0.0
    assert err.max() <= max_tol, "%s: max |err| %.3g (bound %g)" % (what, err.max(), max_tol)
    assert rms <= rms_tol, "%s: rms err %.3g (bound %g)" % (what, rms, rms_tol)
    return float(err.max()), rms


def test_fp8_tiny():
    model, tree, pts = synth.config_tiny()
    m = load(model, tree)
    y_ref, d_ref = oracle.query(model, tree, pts, exit_layers=True)
    y, el = m.query(dev(pts), precision="fp8", exit_layers=True)
    np.testing.assert_array_equal(el.cpu().numpy().astype(np.int32), d_ref)
    check_fp8(y, y_ref, d_ref, "tiny/fp8", fp8_bounds(model))
    m.free()


@pytest.mark.parametrize("tail", [synth.TAIL_LINEAR, synth.TAIL_MULT])
def test_fp8_scene(tail):
    """8 x 256 SIREN on its level-7 octree (64^3 lattice), full depth, LOD clamps, far leaves."""
    model = synth.siren_tmlp(8, 256, seed=1, tail_kind=tail)
    tree = synth.scene_octree(7, 8, far_field=tail == synth.TAIL_MULT)
    m = load(model, tree)
    pts = synth.lattice(64)
    for lod in (0, 3):
        y_ref, d_ref = oracle.query(model, tree, pts, max_depth=lod, exit_layers=True)
        y, el = m.query(dev(pts), precision="fp8", max_depth=lod, exit_layers=True)
        np.testing.assert_array_equal(el.cpu().numpy().astype(np.int32), d_ref)
        check_fp8(y, y_ref, d_ref, "scene64/fp8/lod%d" % lod, fp8_bounds(model))
    full = synth.uniform_points(20001, seed=17)
    check_fp8(m.query(dev(full), precision="fp8", full_depth=True), oracle.full_depth(model, full), None, "full/fp8",
              fp8_bounds(model))
    g = np.random.Generator(np.random.PCG64(3))
    for n in (1, 127, 129, 4097):
        p = g.uniform(-1, 1, (n, 3)).astype(np.float32)
        check_fp8(m.query(dev(p), precision="fp8"), oracle.query(model, tree, p), None, "n=%d" % n, fp8_bounds(model))
    m.free()


def test_fp8_width_336():
    """The wide variant: two MMA column groups and a last K-step half zero padding."""
    model = synth.siren_tmlp(8, 336, seed=2)
    tree = synth.scene_octree(7, 8, transform=synth.rotation([0, 1, 0], 0.5), scale=0.95)
    m = load(model, tree)
    pts = synth.lattice(48)
    y_ref, d_ref = oracle.query(model, tree, pts, exit_layers=True)
    y, el = m.query(dev(pts), precision="fp8", exit_layers=True)
    np.testing.assert_array_equal(el.cpu().numpy().astype(np.int32), d_ref)
    check_fp8(y, y_ref, d_ref, "w336/fp8", fp8_bounds(model))
    full = synth.uniform_points(3001, seed=19)
    check_fp8(m.query(dev(full), precision="fp8", full_depth=True), oracle.full_depth(model, full), None,
              "w336 full/fp8", fp8_bounds(model))
    m.free()


def test_fp8_full_size_sampled():
    """256^3 lattice in the benchmark's launch configuration; error on 20,000 sampled points."""
    model = synth.siren_tmlp(8, 256, seed=1)
    tree = synth.scene_octree(7, 8)
    m = load(model, tree)
    pts = synth.lattice(256)
    y, el = m.query(dev(pts), precision="fp8", exit_layers=True, workspace=m.workspace(len(pts)))
    d_ref, _ = oracle.lookup(tree, pts)
    np.testing.assert_array_equal(el.cpu().numpy().astype(np.int32), d_ref)
    idx = synth.sample_indices(len(pts), 20000, seed=11)
    check_fp8(y.cpu().numpy()[idx], oracle.query(model, tree, pts[idx]), d_ref[idx], "256^3 sampled/fp8",
              fp8_bounds(model))
    m.free()


@pytest.mark.parametrize("tail", [synth.TAIL_LINEAR, synth.TAIL_MULT])
def test_fp8_gradient_full_depth(tail):
    """Tensor-core gradient in FP8 mode: the tangent rows are e4m3-rounded MMA operands like the
    activations.  Bounds: 3x the maximum and 2x the RMS gradient error of the emulation of the
    same rounding (tests/quantised_emulation.py) at full depth on the same 20,000 points
    (8 x 256 SIREN, linear tails: 0.31 / 0.066 of max|g| 2.23; multiplicative: 0.015 / 0.0031).
    Layer 1 is float32 class, so the exit-layer-1 gradient keeps the float32 bound."""
    model = synth.siren_tmlp(8, 256, seed=1, tail_kind=tail)
    max_tol, rms_tol = fp8_bounds(model, grad=True)
    m = load(model)
    pts = synth.uniform_points(20001, seed=17)
    y, g = m.query_grad(dev(pts), precision="fp8", full_depth=True)
    y_ref, g_ref = oracle.full_depth(model, pts, grad=True)
    err = np.abs(g.double().cpu().numpy() - g_ref)
    assert np.isfinite(err).all()
    assert err.max() <= max_tol and np.sqrt((err ** 2).mean()) <= rms_tol, (err.max(), np.sqrt((err ** 2).mean()))
    check_fp8(y, y_ref, None, "grad query value/fp8", fp8_bounds(model))
    tree = synth.scene_octree(7, 8, far_field=tail == synth.TAIL_MULT)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    _, g1 = m.query_grad(dev(pts), precision="fp8", max_depth=1)
    _, g1_ref = oracle.query(model, tree, pts, max_depth=1, grad=True)
    gscale = max(1.0, float(np.abs(g1_ref).max()))
    assert np.abs(g1.double().cpu().numpy() - g1_ref).max() <= 1e-5 * model.omega0 * gscale
    m.free()


def test_fp8_rejects_relu():
    """FP8 stores activations unscaled, valid for the sine's [-1, 1] only: ReLU models are refused."""
    from paper_2604_25936_gb300 import SandError
    model = synth.relu_ff_tmlp(6, 128, n_freq=64, sigma=10.0, seed=3)
    m = load(model)
    with pytest.raises(SandError, match="EUNSUPPORTED"):
        m.query(dev(synth.uniform_points(100, 1)), precision="fp8", full_depth=True)
    m.free()
