"""Depth-map construction on the GPU (sand_build_depth_map, Sec. 3.2, Eq. 5-7) and the
all-tails output it is built on, against the FP64 oracle.

Eq. 5 turns floating-point comparisons into integers.  The float32-class tensor-core
outputs and the float64 oracle can decide differently only where a compared quantity
lies within the output tolerance of its threshold (|y_L - y_i| against r, or a y near 0
for the sign).  Per sample the test derives from the oracle's values the range of depths
such close calls allow, max-pools the ranges per leaf (Eq. 6), and requires every GPU
leaf depth to lie in its leaf's range; leaves whose range is one value (most of them)
must match exactly.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # float32-mode output tolerance


def load(model, tree=None):
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    if tree is not None:
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    return m


def depth_range(ys, r, near, tol=TOL):
    """[lowest, highest] Eq. 5 depth per sample (near: bool per sample) when every decision
    within tol of its threshold may go either way."""
    yl = ys[:, -1:]
    sign_clear = (np.abs(ys) > tol) & (np.abs(yl) > tol)
    same = (ys >= 0) == (yl >= 0)
    diff = np.abs(yl - ys)
    nr = near[:, None]
    sure = same & sign_clear & (~nr | (diff < r - 2 * tol))
    maybe = (same | ~sign_clear) & (~nr | (diff < r + 2 * tol))
    sure[:, -1] = True
    maybe[:, -1] = True
    return np.argmax(maybe, axis=1) + 1, np.argmax(sure, axis=1) + 1


def check_map(m, model, tree, near, k, r, far_sign=False):
    got = m.build_depth_map(tree.max_level, tree.child, near, samples_per_axis=k, r=r, far_sign=far_sign)
    ref, pts, d, rows, ys = oracle.depth_map_from_network(model, tree.child, near, k=k, r=r, far_sign=far_sign)
    cells = oracle.leaf_cells(tree.child)
    cells = cells[[bool(near[c[0]]) or far_sign for c in cells]]
    sample_near = near[cells[rows, 0]].astype(bool)
    lo, hi = depth_range(ys, r, sample_near)
    leaf_lo = np.zeros(len(cells), np.int64)
    leaf_hi = np.zeros(len(cells), np.int64)
    np.maximum.at(leaf_lo, rows, lo)
    np.maximum.at(leaf_hi, rows, hi)
    g = got[cells[:, 0]].astype(np.int64)
    assert ((g >= leaf_lo) & (g <= leaf_hi)).all(), "leaf depth outside the range the tolerance allows"
    fixed = leaf_lo == leaf_hi
    np.testing.assert_array_equal(g[fixed], ref[cells[fixed, 0]])
    assert fixed.mean() > 0.9
    others = np.setdiff1d(np.arange(len(tree.child)), cells[:, 0])
    assert (got[others] == 0).all()
    return got, ref, fixed


def test_all_tails_output():
    model = synth.siren_tmlp(8, 256, seed=1)
    m = load(model)
    pts = synth.uniform_points(20001, seed=41)
    ys = m.query(torch.from_numpy(pts).cuda(), precision="fp32", full_depth=True, all_tails=True)
    _, ref = oracle.evaluate(model, pts, 8, all_tails=True)
    assert ys.shape == (20001, 8)
    err = np.abs(ys.double().cpu().numpy() - ref).max()
    assert err <= TOL, err
    # the last column is the plain full-depth output
    y = m.query(torch.from_numpy(pts).cuda(), precision="fp32", full_depth=True)
    assert torch.equal(y, ys[:, -1])
    m.free()


@pytest.mark.parametrize("r", [1.5e-4, 0.05])
def test_build_siren_map(r):
    model = synth.siren_tmlp(8, 256, seed=1)
    tree = synth.scene_octree(5, 8, far_field=True)
    near = ((tree.child < 0) & (tree.depth > 0)).astype(np.uint8)
    m = load(model)
    check_map(m, model, tree, near, 4, r)
    check_map(m, model, tree, near, 2, r, far_sign=True)
    m.free()


def test_build_sphere_map_and_query():
    """The closed-form ReLU model (y_4 = |p|^2 - R^2): build the map, load it, query with it."""
    model = synth.relu_sphere_tmlp(0.6, width=64)
    tree = synth.voxel_sphere_octree(3, 0.6)
    near = (tree.child < 0).astype(np.uint8)
    m = load(model)
    got, ref, fixed = check_map(m, model, tree, near, 4, 0.2)
    assert len(np.unique(got[tree.child < 0])) > 1  # the closed form gives genuinely different depths
    built = synth.Octree(tree.max_level, tree.n_layers, tree.child, got, tree.far, tree.level, tree.centre)
    m.set_depth_map(built.max_level, built.n_layers, built.child, built.depth, built.far)
    pts = synth.lattice(40)
    y, el = m.query(torch.from_numpy(pts).cuda(), precision="fp32", exit_layers=True)
    y_ref, d_ref = oracle.query(model, built, pts, exit_layers=True)
    np.testing.assert_array_equal(el.cpu().numpy().astype(np.int32), d_ref)
    assert np.abs(y.double().cpu().numpy() - y_ref).max() <= TOL
    m.free()


def test_build_errors():
    from paper_2604_25936_gb300 import SandError
    model = synth.siren_tmlp(8, 256, seed=1)
    tree = synth.scene_octree(4, 8, far_field=True)
    near = ((tree.child < 0) & (tree.depth > 0)).astype(np.uint8)
    m = load(model)
    with pytest.raises(SandError, match="EINVAL"):
        m.build_depth_map(tree.max_level, tree.child, near, samples_per_axis=3)
    with pytest.raises(SandError, match="EINVAL"):
        m.build_depth_map(tree.max_level, tree.child, near, r=0.0)
    bad = tree.child.copy()
    bad[0] = len(bad) - 2
    with pytest.raises(SandError, match="EFORMAT"):
        m.build_depth_map(tree.max_level, bad, near)
    with pytest.raises(SandError, match="EINVAL"):
        m.query(torch.zeros((4, 3), device="cuda"), all_tails=True)  # all_tails needs full_depth
    m.free()
