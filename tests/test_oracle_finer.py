"""The oracle's FINER activation sin(omega0 (|z| + 1) z) — PARITY UNPINNED against the paper.

SAND names the FINER backbone (Sec. 2, the SAND-FINER rows of Table 1) but does not restate
its activation, so nothing in the paper fixes a value.  These tests check what the
mathematics fixes on its own:
* the input gradient against central differences of the oracle's own forward pass;
* the small-argument limit: for |z| << 1/omega0-scale the activation is SIREN's sin(omega0 z)
  up to omega0 z^2, so a FINER and a SIREN network with the same (tiny) weights agree;
* odd symmetry: with zero biases everywhere and linear tails without biases, every
  activation is odd in x, so y(-x) = -y(x) (an even term such as z^2 in place of |z| z fails).
"""
import dataclasses

import numpy as np

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
