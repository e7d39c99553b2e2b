"""Pins of the FP64 oracle against what SAND (arxiv 2604.25936) and mathematics fix.

Each test compares the oracle with something other than itself: exact
rational arithmetic, a float64 PyTorch restatement of Eq. 1 / Eq. 2 built
from library layers, pure-Python loops, closed-form hand-built models, the
quadratic-form identity of Appendix A, and finite differences.  A dropped
term, a wrong sign, a transposed weight or a wrong octant/tie rule in the
oracle fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- restatements
def torch_tmlp(model, pts, depth):
    """Eq. 2 (and Eq. 3) restated with float64 torch.nn.Linear layers; returns y_1..y_depth."""
    x = torch.tensor(np.asarray(pts, np.float64))
    if model.encoder == synth.ENC_FOURIER:
        B = torch.tensor(model.enc_B.astype(np.float64))
        s = 2 * math.pi * (x @ B.T)
        h = torch.cat([torch.sin(s), torch.cos(s)], dim=1)
    else:
        h = x
    ys, y = [], torch.zeros(x.shape[0], dtype=torch.float64)
    for l in range(1, depth + 1):
        W = model.W1 if l == 1 else model.Wh[l - 2]
        b = model.b1 if l == 1 else model.bh[l - 2]
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.tensor(W.astype(np.float64)))
            lin.bias.copy_(torch.tensor(b.astype(np.float64)))
            u = lin(h)
            h = torch.relu(u) if model.activation == synth.ACT_RELU else torch.sin(model.omega0 * u)
            a = torch.tensor(model.tail_w[l - 1, 0].astype(np.float64))
            t = h @ a + float(model.tail_b[l - 1, 0])
            if model.tail_kind == synth.TAIL_MULT and l >= 2:
                bb = torch.tensor(model.tail_w[l - 1, 1].astype(np.float64))
                t = t * (h @ bb + float(model.tail_b[l - 1, 1]))
        y = y + t
        ys.append(y.numpy().copy())
    return np.stack(ys, axis=1)


def exact_cell(x: float, R: int) -> int:
    """floor(x * R / 2) + R / 2 clamped to [0, R-1], in exact rational arithmetic."""
    if math.isinf(x):
        return 0 if x < 0 else R - 1
    q = Fraction(x) * R / 2
    return min(max(math.floor(q) + R // 2, 0), R - 1)


# ------------------------------------------------------------------- lookup pins
def test_tiny_histogram_closed_form():
    """Sec. 3.4 lookup on the 8^3 voxel map equals the voxel formula, counted exactly."""
    gold = json.load(open(os.path.join(GOLD, "tiny_voxel_histogram.json")))
    model, tree, pts = synth.config_tiny()
    d, _ = oracle.lookup(tree, pts)
    hist = np.bincount(d, minlength=5)
    assert {str(k): int(hist[k]) for k in range(1, 5)} == gold["histogram"]
    assert hist[0] == 0
    # independent recount: exact cell index, then the sphere rule at the voxel centre
    R = 8
    cells = {float(v): exact_cell(float(v), R) for v in np.unique(pts)}
    expect = np.empty(len(pts), np.int32)
    for n, p in enumerate(pts):
        c = [-1 + (2 * cells[float(v)] + 1) / R for v in p]
        s = abs(math.sqrt(sum(v * v for v in c)) - 0.5)
        expect[n] = 4 if s < 0.05 else 3 if s < 0.15 else 2 if s < 0.4 else 1
    np.testing.assert_array_equal(d, expect)
    assert abs(d.mean() - gold["mean_exit_layer"]) < 1e-12


@pytest.mark.parametrize("level", [3, 7])
def test_lookup_boundaries_complete_tree(level):
    """Points on, and one ulp either side of, every cell boundary land in the cell
    given by the exact floor formula (upper child on ties, outside clamped)."""
    R = 1 << level
    if level == 3:
        tree = synth.voxel_sphere_octree(3, 0.5)
    else:  # complete level-7 tree whose leaf payload encodes the cell's x index mod 7 + 1
        tree = synth.build_octree(level, 8, lambda c, s, l: np.ones(len(c), bool),
                                  lambda c, s, l: (((np.floor((c[:, 0] + 1) * R / 2)).astype(int) % 7 + 1)
                                                   .astype(np.uint8), c[:, 1].astype(np.float32)))
    pts = synth.boundary_points(level)
    d, far = oracle.lookup(tree, pts)
    for p, dd, ff in zip(pts, d, far):
        i, j, k = (exact_cell(float(v), R) for v in p)
        c = np.array([-1 + (2 * a + 1) / R for a in (i, j, k)])
        if level == 3:
            s = abs(np.linalg.norm(c) - 0.5)
            e = 4 if s < 0.05 else 3 if s < 0.15 else 2 if s < 0.4 else 1
        else:
            e = i % 7 + 1
            assert ff == np.float32(c[1])
        assert dd == e, (p, dd, e)


def test_lookup_adaptive_leaf_contains_point():
    """On the adaptive scene octree the leaf found holds the point in its half-open
    cell [lo, lo + size) (closed at +1), with outside points clamped (exact arithmetic)."""
    tree = synth.scene_octree(7, 8)
    g = np.random.Generator(np.random.PCG64(5))
    pts = np.concatenate([synth.boundary_points(7), g.uniform(-1.2, 1.2, (3000, 3)).astype(np.float32)])
    # locate the leaf by exact containment: for each leaf, its cell bounds
    leaf = np.where(tree.child < 0)[0]
    size = 2.0 / (1 << tree.level[leaf])
    lo = tree.centre[leaf] - size[:, None] / 2
    d, far = oracle.lookup(tree, pts)
    for p, dd, ff in zip(pts, d, far):
        q = np.clip(p.astype(np.float64), -1.0, 1.0)
        inside = np.all((lo <= q) & ((q < lo + size[:, None]) | ((q == 1.0) & (lo + size[:, None] == 1.0))), axis=1)
        hits = leaf[inside]
        assert len(hits) == 1, (p, hits)
        assert dd == tree.depth[hits[0]] and ff == tree.far[hits[0]]


def test_lookup_lod_far_and_nan():
    """LOD clamp (Sec. 3.4) touches only exit layers > max_depth; exit layer 0 returns the
    stored centre value (Eq. 7) with zero gradient; NaN points give -1 / NaN."""
    model = synth.siren_tmlp(8, 32, seed=4)
    tree = synth.scene_octree(5, 8, far_field=True)
    g = np.random.Generator(np.random.PCG64(9))
    pts = g.uniform(-1, 1, (4000, 3)).astype(np.float32)
    pts[7] = [np.nan, 0.0, 0.0]
    pts[11] = [0.1, np.nan, 0.2]
    d_full, far = oracle.lookup(tree, pts)
    assert (d_full == 0).any() and (d_full >= 5).any()
    assert d_full[7] == -1 and d_full[11] == -1 and np.isnan(far[7])
    for k in (1, 3):
        d_k, _ = oracle.lookup(tree, pts, max_depth=k)
        np.testing.assert_array_equal(d_k, np.where(d_full > k, k, d_full))
    y, gr, dq = oracle.query(model, tree, pts, max_depth=3, grad=True, exit_layers=True)
    z = dq == 0
    np.testing.assert_array_equal(y[z], far[z])
    assert np.all(gr[z] == 0.0)
    assert np.isnan(y[7]) and np.isnan(y[11])
    nz = dq > 0
    ye = oracle.evaluate(model, pts[nz], np.minimum(d_full[nz], 3))
    np.testing.assert_array_equal(y[nz], ye)


# ------------------------------------------------------------------- T-MLP pins
@pytest.mark.parametrize("kind", ["siren_linear", "siren_mult", "relu_ff"])
def test_tmlp_matches_torch_layers(kind):
    """Eq. 2 / Eq. 3: every cumulative output y_k equals a float64 torch.nn.Linear restatement."""
    if kind == "siren_linear":
        model = synth.siren_tmlp(5, 48, seed=2)
    elif kind == "siren_mult":
        model = synth.siren_tmlp(5, 48, seed=3, tail_kind=synth.TAIL_MULT)
    else:
        model = synth.relu_ff_tmlp(4, 40, n_freq=16, sigma=3.0, seed=6)
    pts = synth.uniform_points(500, seed=8)
    ref = torch_tmlp(model, pts, model.n_layers)
    y, ys = oracle.evaluate(model, pts, model.n_layers, all_tails=True)
    np.testing.assert_allclose(ys, ref, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(y, ys[:, -1])
    for k in range(1, model.n_layers + 1):   # constant exit layer k returns tail-sum y_k
        np.testing.assert_array_equal(oracle.evaluate(model, pts, k), ys[:, k - 1])


def test_plain_mlp_special_case():
    """Zeroing tails 1..L-1 turns the T-MLP into the plain MLP of Eq. 1, y = W_out h_L + b_out,
    computed here with torch.nn.Sequential (a library model, not a restatement of the oracle)."""
    model = synth.siren_tmlp(6, 32, seed=12)
    model.tail_w[:-1] = 0.0
    model.tail_b[:-1] = 0.0
    w0 = model.omega0

    class Sine(torch.nn.Module):
        def forward(self, u):
            return torch.sin(w0 * u)
    layers = []
    for l in range(model.n_layers):
        W = model.W1 if l == 0 else model.Wh[l - 1]
        b = model.b1 if l == 0 else model.bh[l - 1]
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.tensor(W, dtype=torch.float64))
            lin.bias.copy_(torch.tensor(b, dtype=torch.float64))
        layers += [lin, Sine()]
    out = torch.nn.Linear(model.width, 1).double()
    with torch.no_grad():
        out.weight.copy_(torch.tensor(model.tail_w[-1, 0:1], dtype=torch.float64))
        out.bias.copy_(torch.tensor(model.tail_b[-1, 0:1], dtype=torch.float64))
    mlp = torch.nn.Sequential(*layers, out)
    pts = synth.uniform_points(300, seed=13)
    with torch.no_grad():
        ref = mlp(torch.tensor(pts, dtype=torch.float64)).numpy()[:, 0]
    np.testing.assert_allclose(oracle.full_depth(model, pts), ref, rtol=0, atol=1e-12)


def test_bruteforce_python_loops():
    """Per-point pure-Python evaluation (math.sin, nested loops) on a tiny grid."""
    model = synth.siren_tmlp(3, 12, seed=21, tail_kind=synth.TAIL_MULT)
    pts = synth.lattice(4)
    depth = (np.arange(len(pts)) % 3) + 1
    y = oracle.evaluate(model, pts, depth)
    for n, p in enumerate(pts):
        h = [float(v) for v in p]
        acc = 0.0
        for l in range(1, depth[n] + 1):
            W = model.W1 if l == 1 else model.Wh[l - 2]
            b = model.b1 if l == 1 else model.bh[l - 2]
            h = [math.sin(model.omega0 * (sum(float(W[j][k]) * h[k] for k in range(len(h))) + float(b[j])))
                 for j in range(model.width)]
            t = sum(float(model.tail_w[l - 1][0][j]) * h[j] for j in range(model.width)) + float(model.tail_b[l - 1][0])
            if l >= 2:
                t *= sum(float(model.tail_w[l - 1][1][j]) * h[j] for j in range(model.width)) + float(model.tail_b[l - 1][1])
            acc += t
        assert abs(acc - y[n]) < 1e-13


def test_multiplicative_tail_quadratic_form():
    """Appendix A: (a.h + c)(b.h + d) = h^T (a b^T) h + (d a + c b)^T h + c d, with h the exact
    hidden features of the hand-built ReLU model and of a random SIREN (h from the torch restatement)."""
    pts = synth.uniform_points(200, seed=31)
    # hand-built model: h_l = [x+, x-, y+, y-, z+, z-, 0, 0] exactly
    m = synth.relu_sphere_tmlp(0.5)
    _, ys = oracle.evaluate(m, pts, 4, all_tails=True)
    p = pts.astype(np.float64)
    h = np.stack([np.maximum(p[:, 0], 0), np.maximum(-p[:, 0], 0), np.maximum(p[:, 1], 0),
                  np.maximum(-p[:, 1], 0), np.maximum(p[:, 2], 0), np.maximum(-p[:, 2], 0),
                  np.zeros(len(p)), np.zeros(len(p))], axis=1)
    for l in (2, 3, 4):
        a, b = m.tail_w[l - 1, 0].astype(np.float64), m.tail_w[l - 1, 1].astype(np.float64)
        c, d = float(m.tail_b[l - 1, 0]), float(m.tail_b[l - 1, 1])
        Q, u, s = np.outer(a, b), d * a + c * b, c * d
        t = np.einsum("ni,ij,nj->n", h, Q, h) + h @ u + s
        np.testing.assert_allclose(ys[:, l - 1] - ys[:, l - 2], t, rtol=0, atol=1e-15)
    # random SIREN with multiplicative tails
    m = synth.siren_tmlp(3, 24, seed=32, tail_kind=synth.TAIL_MULT)
    _, ys = oracle.evaluate(m, pts, 3, all_tails=True)
    x = torch.tensor(pts, dtype=torch.float64)
    hh = torch.sin(m.omega0 * (x @ torch.tensor(m.W1, dtype=torch.float64).T + torch.tensor(m.b1, dtype=torch.float64)))
    hh = torch.sin(m.omega0 * (hh @ torch.tensor(m.Wh[0], dtype=torch.float64).T + torch.tensor(m.bh[0], dtype=torch.float64))).numpy()
    a, b = m.tail_w[1, 0].astype(np.float64), m.tail_w[1, 1].astype(np.float64)
    c, d = float(m.tail_b[1, 0]), float(m.tail_b[1, 1])
    t = np.einsum("ni,ij,nj->n", hh, np.outer(a, b), hh) + hh @ (d * a + c * b) + c * d
    np.testing.assert_allclose(ys[:, 1] - ys[:, 0], t, rtol=0, atol=1e-13)


def test_closed_form_sphere_and_plane():
    """Hand-built weights with exact outputs: y1 = -r^2, y2 = x^2 - r^2, y3 = x^2 + y^2 - r^2,
    y4 = |x|^2 - r^2 with gradient 2x (multiplicative tails); plane y1 = n.x - c, gradient n."""
    r = 0.6
    m = synth.relu_sphere_tmlp(r)
    pts = synth.uniform_points(1000, seed=41)
    p = pts.astype(np.float64)
    _, ys = oracle.evaluate(m, pts, 4, all_tails=True)
    np.testing.assert_allclose(ys[:, 0], float(np.float32(-r * r)), rtol=0, atol=0)
    np.testing.assert_allclose(ys[:, 1], p[:, 0] ** 2 + float(np.float32(-r * r)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(ys[:, 2], p[:, 0] ** 2 + p[:, 1] ** 2 + float(np.float32(-r * r)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(ys[:, 3], (p ** 2).sum(1) + float(np.float32(-r * r)), rtol=0, atol=1e-15)
    _, g = oracle.evaluate(m, pts, 4, grad=True)
    np.testing.assert_allclose(g, 2 * p, rtol=0, atol=1e-15)
    n = np.array([0.48, -0.6, 0.64])
    pl = synth.relu_plane_tmlp(n, 0.25)
    y, g = oracle.evaluate(pl, pts, 1, grad=True)
    n32 = n.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(y, p @ n32 - float(np.float32(0.25)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(g, np.broadcast_to(n32, g.shape), rtol=0, atol=0)


@pytest.mark.parametrize("kind", ["siren_linear", "siren_mult", "relu_ff"])
def test_gradient_central_differences(kind):
    """Reverse-mode gradient equals central differences of the oracle's own y_d (step 1e-6 in
    double, truncation ~ h^2 |f'''|)."""
    if kind == "siren_linear":
        model = synth.siren_tmlp(4, 32, seed=51)
    elif kind == "siren_mult":
        model = synth.siren_tmlp(4, 32, seed=52, tail_kind=synth.TAIL_MULT)
    else:
        model = synth.relu_ff_tmlp(3, 32, n_freq=8, sigma=2.0, seed=53)
    pts = synth.uniform_points(64, seed=54).astype(np.float64)
    depth = (np.arange(64) % model.n_layers) + 1
    _, g = oracle.evaluate(model, pts.astype(np.float32), depth, grad=True)
    p32 = pts.astype(np.float32).astype(np.float64)
    # evaluate in double at perturbed points: the oracle takes float32 points, so perturb by
    # exactly representable steps around float32 inputs and use the C routine via torch restatement
    h = 2.0 ** -20
    fd = np.zeros_like(g)
    for a in range(3):
        e = np.zeros(3); e[a] = h
        yp = torch_eval_at(model, p32 + e, depth)
        ym = torch_eval_at(model, p32 - e, depth)
        fd[:, a] = (yp - ym) / (2 * h)
    scale = max(1.0, np.abs(g).max())
    np.testing.assert_allclose(g, fd, rtol=0, atol=2e-6 * scale)


def torch_eval_at(model, pts64, depth):
    ys = torch_tmlp(model, pts64, model.n_layers)
    return ys[np.arange(len(pts64)), np.asarray(depth) - 1]


def test_gradient_matches_torch_autograd():
    """The oracle gradient equals torch.autograd through the float64 restatement."""
    model = synth.siren_tmlp(5, 40, seed=61, tail_kind=synth.TAIL_MULT)
    pts = synth.uniform_points(100, seed=62)
    depth = (np.arange(100) % 5) + 1
    _, g = oracle.evaluate(model, pts, depth, grad=True)
    x = torch.tensor(pts, dtype=torch.float64, requires_grad=True)
    y = torch.zeros(100, dtype=torch.float64)
    h = x
    acc = torch.zeros(100, dtype=torch.float64)
    outs = []
    for l in range(1, 6):
        W = torch.tensor(model.W1 if l == 1 else model.Wh[l - 2], dtype=torch.float64)
        b = torch.tensor(model.b1 if l == 1 else model.bh[l - 2], dtype=torch.float64)
        h = torch.sin(model.omega0 * (h @ W.T + b))
        t = h @ torch.tensor(model.tail_w[l - 1, 0], dtype=torch.float64) + float(model.tail_b[l - 1, 0])
        if l >= 2:
            t = t * (h @ torch.tensor(model.tail_w[l - 1, 1], dtype=torch.float64) + float(model.tail_b[l - 1, 1]))
        acc = acc + t
        outs.append(acc)
    Y = torch.stack(outs, 1)[torch.arange(100), torch.tensor(depth - 1)]
    (gx,) = torch.autograd.grad(Y.sum(), x)
    np.testing.assert_allclose(g, gx.numpy(), rtol=0, atol=1e-11)


def test_preact_margin_closed_form():
    """The hand-built ReLU sphere model (width 6): layer 1's pre-activations are +-x, +-y, +-z,
    so the margin at exit layer 1 is min(|x|, |y|, |z|); layer 2 is the identity on ReLU(+-x, ...),
    half of which are exactly 0, so from layer 2 on the margin is 0; exit layer 0 gives +inf."""
    model = synth.relu_sphere_tmlp(0.6, width=6)
    pts = synth.uniform_points(500, seed=9)
    p = pts.astype(np.float64)
    np.testing.assert_array_equal(oracle.preact_margin(model, pts, 1), np.abs(p).min(1))
    np.testing.assert_array_equal(oracle.preact_margin(model, pts, 3), np.zeros(500))
    d = np.array([0, 1, 2] * 166 + [1, 1], np.int32)
    m = oracle.preact_margin(model, pts, d)
    assert np.isinf(m[d == 0]).all()
    np.testing.assert_array_equal(m[d == 1], np.abs(p[d == 1]).min(1))


def test_preact_margin_brute_force():
    """Against layer-by-layer float64 numpy on a small random ReLU Fourier-feature model."""
    model = synth.relu_ff_tmlp(3, 16, n_freq=8, sigma=2.0, seed=4)
    pts = synth.uniform_points(64, seed=2)
    x = pts.astype(np.float64)
    ph = x @ model.enc_B.astype(np.float64).T
    h = np.concatenate([np.sin(2 * np.pi * ph), np.cos(2 * np.pi * ph)], 1)
    mins = []
    for l in range(3):
        Wl = model.W1 if l == 0 else model.Wh[l - 1]
        bl = model.b1 if l == 0 else model.bh[l - 1]
        u = h @ Wl.astype(np.float64).T + bl.astype(np.float64)
        mins.append(np.abs(u).min(1))
        h = np.maximum(u, 0.0)
    for d in (1, 2, 3):
        np.testing.assert_allclose(oracle.preact_margin(model, pts, d), np.min(mins[:d], 0), rtol=1e-9, atol=1e-12)
