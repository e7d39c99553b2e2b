"""Depth maps deeper than the dense grid (octree levels 8 to 10; the paper's octrees reach depth
9-10, Table 5): the library re-encodes them as a table over the cells of level max_level - 3
whose entries are either a whole leaf or a brick of 8^3 finest cells.  The lookup must still give
every point the exit layer of the oracle's octree descent bit for bit, and far points their
stored value exactly: on every cell boundary of the finest level and one float32 ulp either side
of it, on uniform points, and with the level-of-detail clamp; SDF values within 1e-5.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def tree_of(level, far_field):
    return synth.scene_octree(level, 8, far_field=far_field)


def load(model, tree):
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    return m


@pytest.mark.parametrize("level,far_field", [(8, False), (9, True), (10, False), (10, True)])
def test_deep_map_lookup_is_the_octree_descent(level, far_field):
    model = synth.siren_tmlp(8, 64, seed=61)
    tree = tree_of(level, far_field)
    m = load(model, tree)
    g = np.random.Generator(np.random.PCG64(level))
    pts = np.concatenate([synth.boundary_points(level), g.uniform(-1.1, 1.1, (200000, 3)).astype(np.float32)])
    x = torch.from_numpy(pts).cuda()
    for lod in (0, 3):
        d_ref, f_ref = oracle.lookup(tree, pts, max_depth=lod)
        y, el = m.query(x, precision="fp32_simt", max_depth=lod, exit_layers=True)
        e = el.cpu().numpy().astype(np.int32)
        e[e == 255] = -1
        np.testing.assert_array_equal(e, d_ref)
        far = d_ref == 0
        if far_field:
            assert far.sum() > 1000
        yv = y.cpu().numpy()
        np.testing.assert_array_equal(yv[far], f_ref[far].astype(np.float32))
    # values of network points against the oracle on a sample
    idx = synth.sample_indices(len(pts), 4000, seed=level + 1)
    sane = np.all(np.abs(pts[idx]) <= 100, axis=1)
    y_ref = oracle.query(model, tree, pts[idx][sane])
    y = m.query(torch.from_numpy(np.ascontiguousarray(pts[idx][sane])).cuda(), precision="fp32").double().cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-5
    m.free()


def test_deep_map_rejects_level_11_and_bad_trees():
    from paper_2604_25936_gb300 import SandError
    model = synth.siren_tmlp(2, 64, seed=62)
    tree = tree_of(8, False)
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    with pytest.raises(SandError, match="EUNSUPPORTED"):
        m.set_depth_map(11, tree.n_layers, tree.child, tree.depth, tree.far)
    with pytest.raises(SandError, match="EFORMAT"):  # exit layers beyond the model's 2 layers
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    bad = tree.child.copy()
    inner = np.where(bad >= 0)[0]
    bad[inner[-1]] = 1  # a child link pointing back up the tree
    with pytest.raises(SandError, match="EFORMAT"):
        m.set_depth_map(tree.max_level, tree.n_layers, bad, np.minimum(tree.depth, 2), tree.far)
    m.free()
