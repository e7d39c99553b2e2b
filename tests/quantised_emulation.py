"""Float64 emulation of the tensor-core precision modes — a test helper, not a test.

The 16-bit and FP8 modes of the library round the two operands of every hidden-layer
product (the weights W_l and the activations h_{l-1} of Eq. 2, and in the gradient query
the forward-mode tangents dh_{l-1} / dx) to fp16, bf16 or e4m3 and accumulate in float32.
Their error against the FP64 oracle is therefore an approximation error of the precision,
not a bug, and the GPU tests bound it by this emulation: the same operand rounding, every
other step in float64.

What is rounded, and how (the library's stated packing, independent of its code):
* hidden-layer weights: fp16 after a per-layer power-of-two scale s putting max|W s| in
  [0.5, 1); bf16 unscaled; e4m3 after a per-layer power-of-two scale putting max|W s| in
  [128, 256) (saturating at 448).  A scale is exact, so it is divided out again here.
* activations (and tangents) entering a product: fp16 / bf16 / e4m3 (unscaled, saturating);
* layer 1 on raw coordinates is float32-class on the GPU and exact here; a Fourier-feature
  layer 1 rounds gamma(x) (and its derivative) and W_1 like a hidden layer;
* tails, biases, the sine and the running sums y_l are exact here (float32 on the GPU).
Mode "fp32" rounds nothing, so the emulation must then reproduce the oracle: that is its pin
(tests/test_emulation.py), together with the rounding functions checked bit for bit against
torch's own conversions.

It is numpy arithmetic plus calls of the oracle (the octree lookup and the reference values);
it never calls the CUDA library, and the library never imports it.
"""
from __future__ import annotations

import functools

import numpy as np

import synth

E4M3_MAX = 448.0


def round_f16(a):
    """Nearest fp16 (ties to even), as float64."""
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float64)


def round_bf16(a):
    """Nearest bf16 (ties to even) of the float32 value, as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def round_e4m3(a):
    """Nearest e4m3 value (3 mantissa bits, exponent bias 7, subnormal spacing 2^-9, ties to
    even), saturating at +-448, as float64."""
    x = np.asarray(a, np.float32).astype(np.float64)
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    spacing = np.where(ax >= 2.0 ** -6, np.exp2(e - 3), 2.0 ** -9)
    q = np.round(x / spacing) * spacing   # np.round: ties to even; x / spacing is exact
    return np.clip(q, -E4M3_MAX, E4M3_MAX)


ROUND_ACT = {"fp32": lambda a: np.asarray(a, np.float64), "fp16": round_f16, "bf16": round_bf16, "fp8": round_e4m3}


def round_weights(W, mode):
    """A weight matrix as the mode packs it (scale divided out again)."""
    W = np.asarray(W, np.float32)
    if mode == "fp32":
        return W.astype(np.float64)
    if mode == "bf16":
        return round_bf16(W)
    amax = float(np.abs(W).max())
    if amax == 0.0:
        return np.zeros(W.shape)
    e = np.frexp(np.float32(amax))[1]            # amax = f 2^e, f in [0.5, 1)
    s = 2.0 ** (8 - e) if mode == "fp8" else 2.0 ** (-e)
    scaled = (W.astype(np.float64) * s).astype(np.float32)   # exact: a power of two
    return (round_e4m3(scaled) if mode == "fp8" else round_f16(scaled)) / s


def _act(model, u):
    w0 = model.omega0
    if model.activation == synth.ACT_RELU:
        return np.maximum(u, 0.0), (u > 0).astype(np.float64)
    if model.activation == synth.ACT_FINER:
        p = w0 * (np.abs(u) + 1.0) * u
        return np.sin(p), w0 * (2.0 * np.abs(u) + 1.0) * np.cos(p)
    return np.sin(w0 * u), w0 * np.cos(w0 * u)


def evaluate(model, points, depth, mode: str, grad: bool = False):
    """y_d (float64 [n]) at exit layers `depth` (int or int array; <= 0 gives 0), with the
    operand rounding of `mode`; with grad also dy/dx [n, 3] carried as forward-mode tangents
    whose product operands are rounded like the activations."""
    L, W = model.n_layers, model.width
    x = np.asarray(points, np.float32).reshape(-1, 3).astype(np.float64)
    n = x.shape[0]
    d = np.broadcast_to(np.asarray(depth, np.int64), (n,)).copy()
    d = np.minimum(d, L)
    qa = ROUND_ACT[mode]
    if model.encoder == synth.ENC_FOURIER:
        B = model.enc_B.astype(np.float64)
        s = 2.0 * np.pi * (x @ B.T)
        h0 = np.concatenate([np.sin(s), np.cos(s)], axis=1)
        # d gamma / dx_c: 2 pi B_kc cos(s_k) for the sines, -2 pi B_kc sin(s_k) for the cosines
        dh0 = [np.concatenate([2 * np.pi * B[:, c] * np.cos(s), -2 * np.pi * B[:, c] * np.sin(s)], axis=1)
               for c in range(3)]
        W1 = round_weights(model.W1, mode)
        u = qa(h0) @ W1.T + model.b1.astype(np.float64)
        du = [qa(t) @ W1.T for t in dh0] if grad else None
    else:
        W1 = model.W1.astype(np.float64)
        u = x @ W1.T + model.b1.astype(np.float64)
        du = [np.broadcast_to(W1[:, c], (n, W)).copy() for c in range(3)] if grad else None
    y = np.zeros(n)
    g = np.zeros((n, 3))
    out_y = np.zeros(n)
    out_g = np.zeros((n, 3))
    for l in range(1, L + 1):
        if l > 1:
            Wl = round_weights(model.Wh[l - 2], mode)
            u = qa(h) @ Wl.T + model.bh[l - 2].astype(np.float64)
            if grad:
                du = [qa(t) @ Wl.T for t in dh]
        h, slope = _act(model, u)
        if grad:
            dh = [slope * t for t in du]
        a = model.tail_w[l - 1, 0].astype(np.float64)
        ta = h @ a + float(model.tail_b[l - 1, 0])
        if model.tail_kind == synth.TAIL_MULT and l >= 2:
            b = model.tail_w[l - 1, 1].astype(np.float64)
            tb = h @ b + float(model.tail_b[l - 1, 1])
            t = ta * tb
            if grad:
                dt = np.stack([(t_ @ a) * tb + ta * (t_ @ b) for t_ in dh], axis=1)
        else:
            t = ta
            if grad:
                dt = np.stack([t_ @ a for t_ in dh], axis=1)
        y = y + t
        if grad:
            g = g + dt
        at = d == l
        out_y[at] = y[at]
        if grad:
            out_g[at] = g[at]
        if not (d > l).any():
            break
    return (out_y, out_g) if grad else out_y


@functools.lru_cache(maxsize=None)
def _full_depth_error(key):
    model, mode, grad, n, seed = key
    import oracle
    pts = synth.uniform_points(n, seed=seed)
    if grad:
        y_ref, g_ref = oracle.full_depth(model.value, pts, grad=True)
        y, g = evaluate(model.value, pts, model.value.n_layers, mode, grad=True)
        e = np.abs(g - g_ref)
    else:
        y_ref = oracle.full_depth(model.value, pts)
        e = np.abs(evaluate(model.value, pts, model.value.n_layers, mode) - y_ref)
    return float(e.max()), float(np.sqrt((e ** 2).mean()))


class _Key:
    """Hashable handle of a model (by identity of its parameter bytes) for the cache."""

    def __init__(self, model):
        self.value = model
        self._h = hash((model.header_ints(), model.omega0, model.flat().tobytes()))

    def __hash__(self):
        return self._h

    def __eq__(self, other):
        return isinstance(other, _Key) and self._h == other._h


def full_depth_error(model, mode: str, grad: bool = False, n: int = 20000, seed: int = 17):
    """(max, RMS) error against the FP64 oracle of the emulated mode at full depth on n uniform
    points of [-1, 1]^3 (PCG64 seed): of the values, or with grad of the gradient components."""
    return _full_depth_error((_Key(model), mode, grad, n, seed))


def query(model, octree, points, mode: str, max_depth: int = 0, grad: bool = False):
    """The SAND query (Sec. 3.4) with the operand rounding of `mode`: exit layers and far values
    from the oracle's octree lookup, the network part from evaluate().  NaN points give NaN."""
    import oracle
    d, far = oracle.lookup(octree, points, max_depth=max_depth)
    net = d > 0
    y = np.where(net, 0.0, far)
    g = np.where((d < 0)[:, None], np.nan, 0.0) * np.ones((len(d), 3))
    if net.any():
        pts = np.asarray(points, np.float32).reshape(-1, 3)[net]
        if grad:
            y[net], g[net] = evaluate(model, pts, d[net], mode, grad=True)
        else:
            y[net] = evaluate(model, pts, d[net], mode)
    return (y, g) if grad else y
