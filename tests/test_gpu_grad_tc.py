"""Input gradient on the tensor cores, against the FP64 oracle and central differences.

The tensor-core path evaluates dy/dx by forward-mode tangents in the same pass as the
value: each point takes four rows of a 128-row tile (its value and the three tangents
along x, y, z), the tangent rows go through the same MMAs as the value row, their
pre-activations carry no bias, their activations are cos(u) du (sine) or [u > 0] du (ReLU)
with u the value row's pre-activation, and multiplicative tails (Eq. 3) take the product
rule.  So a tile holds 32 points, and the four rows of one point sit in four consecutive
lanes of one warp.

Tolerances (gradients carry one factor omega0 more than values: each derivative of
sin(omega0 u) multiplies the sensitivity to rounding by omega0):
* float32 split mode: 1e-5 omega0 max|g|, as for the CUDA-core float32 kernel;
* fp16 / bf16 operands: 3x the gradient error, on the same points, of the float64 emulation
  of the same operand rounding (tests/quantised_emulation.py: weights, activations and
  tangents rounded, everything else exact), plus the float32 bound above.  (The value row's
  bound times omega0 would be too loose to catch a wrong term.)
ReLU networks: the gradient jumps where a pre-activation u crosses 0, so a point whose
smallest |u| (the oracle's margin) is within the pre-activation error of 0 may take other
ReLU decisions than the oracle.  The comparison holds on the points whose margin exceeds
1e-4 (float32) or 2^-10 L / 2^-7 L (fp16 / bf16: twice the operand unit roundoff per layer),
and at least 30 such points must remain.
The value outputs of the gradient query and of the plain query (whose layer 1 may run on the
CUDA cores instead) are both held to the oracle at the precision's value tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
import quantised_emulation as qe
import synth

pytestmark = pytest.mark.gpu

# relative pre-activation error per layer of the 16-bit modes (the ReLU decision margin)
REL16 = {"fp16": 2.0 ** -10, "bf16": 2.0 ** -7}
# value tolerances of the parity tests: float32 1e-5, 16-bit 2e-3 (ReLU models in bf16: twice
# the emulated error)
VTOL = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-3}


def load(model, tree=None):
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    if tree is not None:
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def err_of(a, b):
    assert np.array_equal(np.isnan(a), np.isnan(b)), "NaN pattern differs"
    return float(np.abs(np.where(np.isnan(a) & np.isnan(b), 0.0, a - b)).max()) if a.size else 0.0


def grad_tol(model, prec, gscale, emulated_err=0.0):
    w0 = model.omega0 if model.activation == synth.ACT_SINE else 30.0
    if prec == "fp32":
        return 1e-5 * w0 * gscale
    return 3.0 * emulated_err + 1e-5 * w0 * gscale


def model_of(kind):
    if kind == "siren":
        return synth.siren_tmlp(8, 256, seed=1), synth.scene_octree(7, 8)
    if kind == "siren_mult":
        return synth.siren_tmlp(8, 256, seed=1, tail_kind=synth.TAIL_MULT), synth.scene_octree(7, 8, far_field=True)
    if kind == "siren_w64":
        return synth.siren_tmlp(4, 64, seed=2), synth.scene_octree(6, 4, far_field=True)
    if kind == "siren_w336":
        return synth.siren_tmlp(8, 336, seed=2), synth.scene_octree(7, 8, transform=synth.rotation([0, 1, 0], 0.5),
                                                                    scale=0.95)
    return synth.relu_ff_tmlp(6, 128, n_freq=64, sigma=10.0, seed=3), synth.scene_octree(7, 6)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("kind", ["siren", "siren_mult", "siren_w64", "siren_w336", "relu_ff"])
def test_tc_gradient_parity(kind, prec):
    """SAND queries (depth map, binned by exit layer, tiles straddling two bins, a ragged last
    tile of 6001 or 20001 mod 32 points) against the oracle value and gradient."""
    model, tree = model_of(kind)
    m = load(model, tree)
    pts = synth.uniform_points(20001 if model.activation == synth.ACT_RELU else 6001, seed=23)
    y_ref, g_ref, d_ref = oracle.query(model, tree, pts, grad=True, exit_layers=True)
    y, g, el = m.query_grad(dev(pts), precision=prec, exit_layers=True)
    np.testing.assert_array_equal(el.cpu().numpy(), d_ref)
    y = y.double().cpu().numpy()
    g = g.double().cpu().numpy()
    gscale = max(1.0, float(np.abs(g_ref).max()))
    keep = np.ones(len(pts), bool)
    if model.activation == synth.ACT_RELU:
        delta = 1e-4 if prec == "fp32" else REL16[prec] * model.n_layers
        keep = oracle.preact_margin(model, pts, np.maximum(d_ref, 0)) > delta
        assert keep.sum() >= 30, keep.sum()
    e = err_of(g[keep].ravel(), g_ref[keep].ravel())
    e_emu = 0.0
    if prec != "fp32":
        y_emu, g_emu = qe.query(model, tree, pts, prec, grad=True)
        e_emu = err_of(g_emu[keep].ravel(), g_ref[keep].ravel())
    tol = grad_tol(model, prec, gscale, e_emu)
    print("tc-grad %s/%s: %d points, max|g| %.3g  err %.3g  tol %.3g  (%.2e of max|g|)"
          % (kind, prec, keep.sum(), gscale, e, tol, e / gscale))
    assert e <= tol, (kind, prec, e, tol)
    # values of the gradient query and of the plain query (whose layer 1 may run on the CUDA
    # cores) against the oracle, at the precision's value tolerance
    y_plain = m.query(dev(pts), precision=prec).double().cpu().numpy()
    vscale = max(1.0, float(np.abs(y_ref).max()))
    relu_bf16 = model.activation == synth.ACT_RELU and prec == "bf16"
    # ReLU activations are unbounded: in bf16 twice the emulated error instead of the 2e-3 bar
    vtol = 2.0 * err_of(y_emu, y_ref) if relu_bf16 else VTOL[prec] * vscale
    assert err_of(y, y_ref) <= vtol and err_of(y_plain, y_ref) <= vtol, (err_of(y, y_ref), err_of(y_plain, y_ref), vtol)
    m.free()


def test_tc_gradient_vs_central_differences():
    """float32 split mode on the 8 x 256 SIREN, against central differences of the oracle
    at float32-representable steps (h = 1e-4) on 400 network points."""
    model, tree = model_of("siren")
    m = load(model, tree)
    pts = synth.uniform_points(3000, seed=31)
    y_ref, g_ref, d_ref = oracle.query(model, tree, pts, grad=True, exit_layers=True)
    _, g = m.query_grad(dev(pts), precision="fp32")
    g = g.double().cpu().numpy()
    gscale = max(1.0, float(np.abs(g_ref).max()))
    w0 = model.omega0
    net = np.where(d_ref > 0)[0][:400]
    fd = np.zeros((len(net), 3))
    for a in range(3):
        pp, pm = pts[net].copy(), pts[net].copy()
        pp[:, a] += np.float32(1e-4)
        pm[:, a] -= np.float32(1e-4)
        step = pp[:, a].astype(np.float64) - pm[:, a].astype(np.float64)
        fd[:, a] = (oracle.evaluate(model, pp, d_ref[net]) - oracle.evaluate(model, pm, d_ref[net])) / step
    trunc = 1e-4 ** 2 * w0 ** 3 * gscale  # |f'''| h^2 bound for a sine network
    assert err_of(g[net].ravel(), fd.ravel()) <= 1e-5 * w0 * gscale + trunc
    m.free()


def test_tc_gradient_closed_form_sphere():
    """Hand-built ReLU model with multiplicative tails: y_4 = |x|^2 - R^2, gradient 2x, at full
    depth; the product rule of Eq. 3 is the only route to a non-zero gradient."""
    model = synth.relu_sphere_tmlp(0.6, width=64)
    m = load(model)
    pts = synth.uniform_points(3000, seed=5)
    p = pts.astype(np.float64)
    y, g = m.query_grad(dev(pts), precision="fp32", full_depth=True)
    assert err_of(y.double().cpu().numpy(), (p ** 2).sum(1) + float(np.float32(-0.36))) <= 2e-6
    assert err_of(g.double().cpu().numpy().ravel(), (2 * p).ravel()) <= 2e-6
    m.free()


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 4097])
def test_tc_gradient_sizes(n):
    """Empty input, one point, one tile exactly, one point over, a ragged multi-tile count;
    full depth, float32 split mode."""
    model = synth.siren_tmlp(4, 64, seed=2)
    m = load(model)
    pts = synth.uniform_points(max(n, 1), seed=7)[:n]
    y, g = m.query_grad(dev(pts).reshape(n, 3), precision="fp32", full_depth=True)
    assert y.shape == (n,) and g.shape == (n, 3)
    if n:
        y_ref, g_ref = oracle.full_depth(model, pts, grad=True)
        gscale = max(1.0, float(np.abs(g_ref).max()))
        assert err_of(y.double().cpu().numpy(), y_ref) <= 1e-5
        assert err_of(g.double().cpu().numpy().ravel(), g_ref.ravel()) <= 1e-5 * model.omega0 * gscale
    m.free()


def test_tc_autograd():
    from paper_2604_25936_gb300 import SandSDF
    model, tree = model_of("siren")
    m = load(model, tree)
    pts = synth.uniform_points(777, seed=29)
    x = dev(pts).requires_grad_(True)
    y = SandSDF.apply(x, m, "fp32")
    w = torch.linspace(-1, 1, 777, device="cuda")
    (y * w).sum().backward()
    _, g_ref = oracle.query(model, tree, pts, grad=True)
    gscale = max(1.0, float(np.abs(g_ref).max()))
    assert err_of(x.grad.double().cpu().numpy().ravel(), (g_ref * np.linspace(-1, 1, 777)[:, None]).ravel()) \
        <= 1e-5 * model.omega0 * gscale
    m.free()


def test_tc_gradient_without_values():
    """Full-depth gradient query with d_out = NULL through the C-ABI: only the gradient is written."""
    import ctypes
    from paper_2604_25936_gb300 import binding
    model = synth.siren_tmlp(4, 64, seed=2)
    m = load(model)
    pts = synth.uniform_points(300, seed=3)
    g = torch.full((300, 3), float("nan"), device="cuda")
    x = dev(pts)
    o = m._opts("fp32", 0, True, None, None)
    rc = binding.lib().sand_query_sdf_grad(m._h, ctypes.c_void_p(x.data_ptr()), 300, None, ctypes.c_void_p(g.data_ptr()),
                                           ctypes.byref(o), None)
    torch.cuda.synchronize()
    assert rc == 0
    _, g_ref = oracle.full_depth(model, pts, grad=True)
    gscale = max(1.0, float(np.abs(g_ref).max()))
    assert err_of(g.double().cpu().numpy().ravel(), g_ref.ravel()) <= 1e-5 * model.omega0 * gscale
    m.free()
