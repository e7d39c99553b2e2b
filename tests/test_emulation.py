"""Pins of the float64 precision-mode emulation (tests/quantised_emulation.py) that the GPU
tests take their 16-bit and FP8 bounds from.

* Its rounding functions agree bit for bit with torch's own fp16, bf16 and float8_e4m3fn
  conversions (ties, subnormals and the e4m3 saturation at 448 included).
* With nothing rounded (mode "fp32") it reproduces the FP64 oracle, values and gradients,
  for every activation, tail kind and encoder, at mixed exit layers: the emulation computes
  Eq. 2 / Eq. 3 itself, so a slip there (a dropped tail, a wrong tangent) fails here.
* Rounding only the weights moves the result by the amount the packing rule implies: a
  per-layer power-of-two scale is exact, so e4m3 weights scaled into [128, 256) lose
  exactly what e4m3 rounding of the scaled values loses.
"""
import numpy as np
import pytest
import torch

import oracle
import quantised_emulation as qe
import synth


def _samples(n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    a = (g.standard_normal(n) * np.exp2(g.uniform(-14, 9, n))).astype(np.float32)
    # exact ties of each format and values at the subnormal boundaries
    ties = np.array([1 + 2.0 ** -4, 1 + 3 * 2.0 ** -4, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -11,
                     1 + 3 * 2.0 ** -11, 2.0 ** -6, 2.0 ** -7, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -14, 2.0 ** -24,
                     0.0, 448.0, 447.9, 240.0, 248.0], np.float32)
    return np.concatenate([a, ties, -ties])


def test_rounding_matches_torch_conversions():
    a = _samples(200000, 1)
    t = torch.from_numpy(a)
    np.testing.assert_array_equal(qe.round_f16(a), t.to(torch.float16).double().numpy())
    np.testing.assert_array_equal(qe.round_bf16(a), t.to(torch.bfloat16).double().numpy())
    inr = a[np.abs(a) <= 448]
    np.testing.assert_array_equal(qe.round_e4m3(inr), torch.from_numpy(inr).to(torch.float8_e4m3fn).double().numpy())
    # saturation (the library converts with SATFINITE): beyond 448 stays at +-448
    np.testing.assert_array_equal(qe.round_e4m3(np.array([500.0, -1e6, 449.0], np.float32)), [448.0, -448.0, 448.0])


MODELS = {
    "siren": lambda: synth.siren_tmlp(6, 32, seed=5),
    "siren_mult": lambda: synth.siren_tmlp(6, 32, seed=6, tail_kind=synth.TAIL_MULT),
    "finer": lambda: synth.finer_tmlp(5, 24, seed=7),
    "relu_ff": lambda: synth.relu_ff_tmlp(4, 32, n_freq=16, sigma=4.0, seed=8),
}


@pytest.mark.parametrize("kind", sorted(MODELS))
def test_unrounded_emulation_is_the_oracle(kind):
    model = MODELS[kind]()
    pts = synth.uniform_points(700, seed=9)
    depth = np.random.Generator(np.random.PCG64(10)).integers(1, model.n_layers + 1, len(pts))
    y_ref, g_ref = oracle.evaluate(model, pts, depth, grad=True)
    y, g = qe.evaluate(model, pts, depth, "fp32", grad=True)
    ys = max(1.0, float(np.abs(y_ref).max()))
    gs = max(1.0, float(np.abs(g_ref).max()))
    assert np.abs(y - y_ref).max() <= 1e-12 * ys
    assert np.abs(g - g_ref).max() <= 1e-11 * gs
    np.testing.assert_array_equal(qe.evaluate(model, pts, depth, "fp32"), y)


def test_weight_packing_scale_is_exact():
    """e4m3 with a power-of-two scale: W s lands in [128, 256) at its maximum, and dividing the
    rounded values by s gives values whose relative error is at most 2^-4 (3 mantissa bits)
    for every weight in the normal range."""
    W = synth.siren_tmlp(3, 64, seed=11).Wh[0]
    q = qe.round_weights(W, "fp8")
    e = np.frexp(np.float32(np.abs(W).max()))[1]
    s = 2.0 ** (8 - e)
    assert 128 <= np.abs(W).max() * s < 256
    normal = np.abs(W) * s >= 2.0 ** -6
    assert (np.abs(q - W)[normal] <= 2.0 ** -4 * np.abs(W)[normal]).all()
    np.testing.assert_array_equal(q * s, qe.round_e4m3((W.astype(np.float64) * s).astype(np.float32)))
    q16 = qe.round_weights(W, "fp16")
    assert (np.abs(q16 - W) <= 2.0 ** -11 * np.abs(W) + 2.0 ** -25).all()


def test_emulated_errors_are_the_precision_not_the_arithmetic():
    """The emulated error of each mode shrinks with the operand precision (fp16 < bf16 < e4m3)
    and is 0 without rounding; printed for the record of the GPU tests' bounds."""
    model = synth.siren_tmlp(8, 64, seed=12)
    errs = {m: qe.full_depth_error(model, m, n=2000) for m in ("fp32", "fp16", "bf16", "fp8")}
    print({m: "%.3g / %.3g" % e for m, e in errs.items()})
    assert errs["fp32"][0] <= 1e-12
    assert errs["fp16"][0] < errs["bf16"][0] < errs["fp8"][0]
