"""FINER backbone (variable-periodic sine sin(omega0 (|z| + 1) z)) through the C-ABI, against
the FP64 oracle.  SAND cites FINER without restating its activation; the oracle's FINER is
pinned to FINER's published definition, evaluated in 50-digit arithmetic
(tests/test_oracle_finer.py); these tests hold the CUDA paths to that oracle.

Tolerances: values as for SIREN (1e-5 float32, 2e-3 16-bit); float32 gradients 1e-5 omega0
max|g| scaled by the activation's larger slope omega0 (2 |z| + 1) <= 5 omega0 for the |z| <= 2
of these models; 16-bit gradients 3x the error of the float64 emulation of the same operand
rounding on the same points (tests/quantised_emulation.py) plus that float32 bound; FP8 values
at full depth 3x the emulated maximum error.  Exit layers bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import quantised_emulation as qe
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp32_simt": 1e-5, "fp16": 2e-3, "bf16": 2e-3}


def load(model, tree=None):
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    if tree is not None:
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt", "fp16", "bf16"])
@pytest.mark.parametrize("tail", [synth.TAIL_LINEAR, synth.TAIL_MULT])
def test_finer_sand_query(tail, prec):
    model = synth.finer_tmlp(8, 256, seed=1, tail_kind=tail)
    tree = synth.scene_octree(7, 8, far_field=tail == synth.TAIL_MULT)
    m = load(model, tree)
    pts = synth.uniform_points(6001, seed=23)
    y_ref, g_ref, d_ref = oracle.query(model, tree, pts, grad=True, exit_layers=True)
    y, el = m.query(dev(pts), precision=prec, exit_layers=True)
    np.testing.assert_array_equal(el.cpu().numpy().astype(np.int32), d_ref)
    vscale = max(1.0, float(np.abs(y_ref).max()))
    err = float(np.abs(y.double().cpu().numpy() - y_ref).max())
    print("finer %s/%d value err %.3g" % (prec, tail, err))
    assert err <= TOL[prec] * vscale, err
    yg, g = m.query_grad(dev(pts), precision=prec)
    gscale = max(1.0, float(np.abs(g_ref).max()))
    gerr = float(np.abs(g.double().cpu().numpy() - g_ref).max())
    gtol = 1e-5 * 5 * model.omega0 * gscale
    if not prec.startswith("fp32"):
        _, g_emu = qe.query(model, tree, pts, prec, grad=True)
        gtol += 3.0 * float(np.abs(g_emu - g_ref).max())
    print("finer %s/%d grad err %.3g (max|g| %.3g, tol %.3g)" % (prec, tail, gerr, gscale, gtol))
    assert gerr <= gtol, (gerr, gtol)
    m.free()


def test_finer_fp8_and_full_depth():
    model = synth.finer_tmlp(8, 256, seed=1)
    m = load(model)
    pts = synth.uniform_points(20001, seed=17)
    y_ref = oracle.full_depth(model, pts)
    fp8_tol = 3.0 * qe.full_depth_error(model, "fp8")[0]
    for prec, tol in (("fp32", 1e-5 * max(1.0, float(np.abs(y_ref).max()))), ("fp8", fp8_tol)):
        y = m.query(dev(pts), precision=prec, full_depth=True).double().cpu().numpy()
        err = float(np.abs(y - y_ref).max())
        print("finer full depth %s err %.3g (bound %.3g)" % (prec, err, tol))
        assert err <= tol, (prec, err, tol)
    m.free()
