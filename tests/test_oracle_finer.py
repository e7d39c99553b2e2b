"""The oracle's FINER activation sin(omega0 (|z| + 1) z).

SAND names the FINER backbone (Sec. 2, the SAND-FINER rows of Table 1) but does not restate
its activation, so the paper itself fixes no value; the oracle follows FINER's published
definition, and the last test pins it there: hand-set width-1 layers put the pre-activations
at chosen values, and y and dy/dx must equal the definition evaluated in 50-digit arithmetic.
The other tests check what the mathematics fixes on its own:
* the input gradient against central differences of the oracle's own forward pass;
* the small-argument limit: for |z| << 1/omega0-scale the activation is SIREN's sin(omega0 z)
  up to omega0 z^2, so a FINER and a SIREN network with the same (tiny) weights agree;
* odd symmetry: with zero biases everywhere and linear tails without biases, every
  activation is odd in x, so y(-x) = -y(x) (an even term such as z^2 in place of |z| z fails).
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth


def test_finer_gradient_central_differences():
    model = synth.finer_tmlp(4, 32, seed=3)
    pts = synth.uniform_points(200, seed=4)
    y, g = oracle.full_depth(model, pts, grad=True)
    h = 1e-6
    for a in range(3):
        pp, pm = pts.astype(np.float64).copy(), pts.astype(np.float64).copy()
        pp[:, a] += h
        pm[:, a] -= h
        # the oracle widens float32 inputs: step in float64 through a float32-exact lattice
        pp32, pm32 = pp.astype(np.float32), pm.astype(np.float32)
        step = pp32[:, a].astype(np.float64) - pm32[:, a].astype(np.float64)
        fd = (oracle.full_depth(model, pp32) - oracle.full_depth(model, pm32)) / step
        gs = max(1.0, float(np.abs(g).max()))
        assert np.abs(fd - g[:, a]).max() <= 1e-3 * gs, np.abs(fd - g[:, a]).max()


def test_finer_small_argument_limit_is_siren():
    base = synth.finer_tmlp(3, 16, seed=5)
    tiny = dataclasses.replace(base, W1=(base.W1 * 1e-4).astype(np.float32), b1=np.zeros_like(base.b1),
                               Wh=(base.Wh * 1e-2).astype(np.float32), bh=np.zeros_like(base.bh))
    siren = dataclasses.replace(tiny, activation=synth.ACT_SINE)
    pts = synth.uniform_points(500, seed=6)
    yf, gf = oracle.full_depth(tiny, pts, grad=True)
    ys, gs = oracle.full_depth(siren, pts, grad=True)
    # |z| <= 1e-4 (|W1| <= 1e-4 / 3, |x| <= 1, three inputs; the hidden layers' z are smaller
    # still): sin(omega0 (|z| + 1) z) = sin(omega0 z) (1 + O(|z|)), so the outputs agree to a
    # relative 1e-4, and the slopes omega0 (2 |z| + 1) cos(.) to 2e-4; bounds with a factor 3
    assert np.abs(yf - ys).max() <= 3e-4 * np.abs(ys).max()
    assert np.abs(gf - gs).max() <= 6e-4 * np.abs(gs).max()
    assert np.abs(yf - ys).max() > 0  # the two activations do differ


def test_finer_odd_symmetry():
    base = synth.finer_tmlp(4, 32, seed=7)
    odd = dataclasses.replace(base, b1=np.zeros_like(base.b1), bh=np.zeros_like(base.bh),
                              tail_b=np.zeros_like(base.tail_b))
    pts = synth.uniform_points(300, seed=8)
    y_pos = oracle.full_depth(odd, pts)
    y_neg = oracle.full_depth(odd, -pts)
    assert np.abs(y_pos + y_neg).max() <= 1e-12 * max(1.0, np.abs(y_pos).max())
    assert np.abs(y_pos).max() > 1e-3


def _finer_chain(w1x, b1, w2, b2, omega0):
    """A FINER T-MLP of width 1 whose first unit sees z1 = w1x * x + b1: two layers, unit tail
    weights, no tail biases.  Returns the model (parameters exact in float32)."""
    L, W = 2, 1
    return synth.TMLP(L, W, 3, synth.TAIL_LINEAR, synth.ACT_FINER, synth.ENC_NONE, 0, float(omega0), None,
                      np.array([[w1x, 0.0, 0.0]], np.float32), np.array([b1], np.float32),
                      np.array([[[w2]]], np.float32), np.array([b2], np.float32),
                      np.array([[[1.0], [0.0]], [[1.0], [0.0]]], np.float32), np.zeros((L, 2), np.float32))


def test_finer_matches_its_definition():
    """FINER (Liu et al., CVPR 2024) defines its activation as sin(omega0 (|z| + 1) z).  With
    hand-set width-1 layers the pre-activations take chosen values (negative, |z| near 0.5,
    near 0, beyond 1), and the oracle's y_1, y_2 and dy_2/dx must equal that definition
    evaluated in 50-digit arithmetic (mpmath; the derivative by mpmath's own numerical
    differentiation, not by a derivative formula).  Plausible misreadings, e.g.
    sin(omega0 (z^2 + 1) z) or sin(omega0 (|z| + 1)) z, differ from it here by far more than
    the 1e-12 allowed (checked below), so they fail."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    w0 = 30.0
    w1x, b1, w2, b2 = 1.0, 0.0, 0.5, 0.25
    model = _finer_chain(w1x, b1, w2, b2, w0)
    xs = np.array([-0.9, -0.5, -0.3125, -0.0625, 0.015625, 0.125, 0.5, 0.75, 0.96875], np.float32)
    pts = np.stack([xs, np.full_like(xs, 0.25), np.full_like(xs, -0.5)], axis=1)
    y, g, ys = oracle.evaluate(model, pts, 2, grad=True, all_tails=True)

    def act(z, form="finer"):
        if form == "finer":
            return mpmath.sin(w0 * (abs(z) + 1) * z)
        if form == "square":
            return mpmath.sin(w0 * (z * z + 1) * z)
        return mpmath.sin(w0 * (abs(z) + 1)) * z

    def y2(x, form="finer"):
        h1 = act(mpmath.mpf(w1x) * x + b1, form)
        h2 = act(mpmath.mpf(w2) * h1 + b2, form)
        return h1, h1 + h2

    for i, xf in enumerate(xs):
        x = mpmath.mpf(float(xf))
        h1, yy = y2(x)
        assert abs(ys[i, 0] - float(h1)) <= 1e-12
        assert abs(y[i] - float(yy)) <= 1e-12
        dydx = mpmath.diff(lambda t: y2(t)[1], x)
        assert abs(g[i, 0] - float(dydx)) <= 1e-9 * max(1.0, abs(float(dydx)))
        assert g[i, 1] == 0.0 and g[i, 2] == 0.0
    for form in ("square", "outer"):
        diff = max(abs(float(y2(mpmath.mpf(float(xf)), form)[1] - y2(mpmath.mpf(float(xf)))[1])) for xf in xs)
        assert diff > 1e-3, (form, diff)
