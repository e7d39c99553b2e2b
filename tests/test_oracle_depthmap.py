"""Pins of the oracle's construction of the network-depth map (Sec. 3.2, Eq. 5-7).

* leaf enumeration against the octree generator's own record of levels and centres;
* the sample lattice: cell centres at k = 1, containment, exactness in float32;
* Eq. 5 on the hand-built ReLU model whose cumulative outputs are known in closed
  form (y_1 = -R^2, y_2 = x^2 - R^2, y_3 = x^2 + y^2 - R^2, y_4 = |p|^2 - R^2), with the
  depths worked out by hand from the equation's text;
* Eq. 6 against a brute-force per-leaf, per-sample loop on a small tree.
"""
import numpy as np
import pytest

import oracle
import synth


def test_leaf_cells_match_generator():
    tree = synth.scene_octree(5, 8, far_field=True)
    cells = oracle.leaf_cells(tree.child)
    assert sorted(cells[:, 0].tolist()) == sorted(np.where(tree.child < 0)[0].tolist())
    for node, lv, ix, iy, iz in cells:
        assert tree.level[node] == lv
        side = 2.0 / 2 ** lv
        np.testing.assert_array_equal(tree.centre[node], -1.0 + (np.array([ix, iy, iz]) + 0.5) * side)
    assert sum((2.0 / 2 ** c[1]) ** 3 for c in cells) == 8.0  # the leaves tile the domain


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_leaf_samples(k):
    tree = synth.scene_octree(4, 8)
    cells = oracle.leaf_cells(tree.child)
    pts = oracle.leaf_samples(cells, k).astype(np.float64).reshape(len(cells), k ** 3, 3)
    side = 2.0 / np.exp2(cells[:, 1])
    lo = -1.0 + cells[:, 2:5] * side[:, None]
    assert ((pts > lo[:, None, :]) & (pts < (lo + side[:, None])[:, None, :])).all()
    if k == 1:
        np.testing.assert_array_equal(pts[:, 0, :], tree.centre[cells[:, 0]])
    # distinct points, spaced side / k apart along x (x fastest)
    if k > 1:
        np.testing.assert_array_equal(pts[:, 1, 0] - pts[:, 0, 0], side / k)
    # exact: the float32 values equal the real-number lattice
    exact = lo[:, None, :] + (np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij")[::-1], -1).reshape(-1, 3)[None]
                              + 0.5) * (side / k)[:, None, None]
    np.testing.assert_array_equal(pts, exact)


def _sphere_outputs(p, R):
    x, y, z = p
    return [-R * R, x * x - R * R, x * x + y * y - R * R, x * x + y * y + z * z - R * R]


@pytest.mark.parametrize("p,R,r,near,expect", [
    ((0.5, 0.0, 0.0), 0.6, 1e-2, True, 2),    # y = (-.36, -.11, -.11, -.11): y_2 = y_L, same sign
    ((0.5, 0.5, 0.0), 0.6, 1e-2, True, 3),    # y = (-.36, -.11, .14, .14): y_2 has the wrong sign
    ((0.1, 0.1, 0.1), 0.6, 1.5e-2, True, 3),  # |y_L - y_i| = .03, .02, .01, 0: first below r at i = 3
    ((0.1, 0.1, 0.1), 0.6, 5e-3, True, 4),    # ... and only i = 4 below 5e-3
    ((0.1, 0.1, 0.1), 0.6, 5e-3, False, 1),   # far leaf: the sign alone, all negative
    ((0.5, 0.0, 0.0), 0.5, 1e-2, True, 2),    # y_L = 0 counts as positive: y_1 = -.25 is not
    ((0.5, 0.0, 0.0), 0.5, 1e-2, False, 2),
    ((0.0, 0.0, 0.9), 0.6, 1e-2, False, 4),   # y_1..y_3 = -.36, y_4 = .45
])
def test_required_depth_closed_form(p, R, r, near, expect):
    model = synth.relu_sphere_tmlp(R, width=8)
    _, ys = oracle.evaluate(model, np.array([p], np.float32), 4, all_tails=True)
    pf = np.array(p, np.float32).astype(np.float64)
    np.testing.assert_allclose(ys[0], _sphere_outputs(pf, R), atol=1e-6)
    assert oracle.required_depth(ys, r, near)[0] == expect


def test_depth_map_brute_force():
    """Eq. 6 on a small tree: a plain loop over leaves and samples, Eq. 5 read literally."""
    model = synth.siren_tmlp(4, 64, seed=0)
    tree = synth.scene_octree(3, 4, far_field=True)
    near = (tree.child < 0) & (tree.depth > 0)
    r = 0.02
    for far_sign in (False, True):
        depth, pts, d, rows, ys = oracle.depth_map_from_network(model, tree.child, near, k=2, r=r, far_sign=far_sign)
        expect = np.zeros(len(tree.child), np.uint8)
        for node in np.where(tree.child < 0)[0]:
            if not near[node] and not far_sign:
                continue
            side = 2.0 / 2 ** tree.level[node]
            best = 0
            for sx in range(2):
                for sy in range(2):
                    for sz in range(2):
                        q = tree.centre[node] - side / 2 + (np.array([sx, sy, sz]) + 0.5) * side / 2
                        _, yq = oracle.evaluate(model, q[None].astype(np.float32), 4, all_tails=True)
                        yq = yq[0]
                        sgn = lambda v: 1 if v >= 0 else -1
                        di = 4
                        for i in range(1, 5):
                            if sgn(yq[i - 1]) == sgn(yq[3]) and (not near[node] or abs(yq[3] - yq[i - 1]) < r):
                                di = i
                                break
                        best = max(best, di)
            expect[node] = best
        np.testing.assert_array_equal(depth, expect)


@pytest.mark.parametrize("p,R,r,expect_layer,expect_y", [
    ((0.05, 0.5, 0.0), 0.6, 1e-2, 2, 0.05 ** 2 - 0.36),          # t = (-.36, .0025, .25, 0): stops at 2
    ((0.5, 0.05, 0.5), 0.6, 1e-2, 3, 0.25 + 0.0025 - 0.36),      # t_3 = .0025
    ((0.5, 0.5, 0.5), 0.6, 1e-2, 4, 0.75 - 0.36),                # no tail below r: layer L
    ((0.5, 0.5, 0.5), 0.05, 1e-2, 1, -0.0025),                   # |t_1| = R^2 = .0025 < r: layer 1
])
def test_dynamic_exit_closed_form(p, R, r, expect_layer, expect_y):
    """Table 6's dynamic exit on the hand-built model, whose tails are -R^2, x^2, y^2, z^2."""
    model = synth.relu_sphere_tmlp(R, width=8)
    y, d, _ = oracle.dynamic_exit(model, np.array([p], np.float32), r)
    assert d[0] == expect_layer
    assert abs(y[0] - expect_y) < 1e-6
