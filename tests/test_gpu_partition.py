"""The row partition of a SAND query between the tensor-core pipeline and the CUDA-core warps,
checked on the kernel itself (tests/test_schedule_host.py checks a host restatement of the
same index arithmetic).

Rows are sorted by descending exit layer; rows [0, bin_start[1]) go through the tensor-core
tiles, rows [bin_start[1], n) (exit layer 1) through the CUDA-core warps of the same kernel.
A one-level octree gives exit layer 2 to the octant x, y, z < 0 and 1 elsewhere, so placing
k points in that octant puts bin_start[1] exactly at k.  With the output prefilled with NaN,
every point must come back finite and equal to the oracle: a row that neither side wrote, or
that one side wrote with the other's layer count, fails.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": 2e-3, "fp32_simt": 1e-5}


def octant_tree(n_layers):
    return synth.build_octree(1, n_layers, lambda c, side, lev: np.ones(len(c), bool),
                              lambda c, side, lev: (np.where((c < 0).all(axis=1), 2, 1).astype(np.uint8),
                                                    np.zeros(len(c), np.float32)))


def points(n, k, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    inner = g.uniform(-0.99, -0.01, (k, 3))
    outer = g.uniform(-0.99, 0.99, (n - k, 3))
    outer[:, 0] = np.abs(outer[:, 0]) + 0.005  # x > 0: never the exit-layer-2 octant
    p = np.concatenate([inner, outer])[g.permutation(n)]
    return p.astype(np.float32)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("n,k", [(1000, 0), (1000, 127), (1000, 128), (1000, 129), (1000, 1000), (1, 1), (1, 0),
                                 (155725, 19457), (155725, 19456)])
def test_partition_covers_every_row(prec, n, k):
    model = synth.siren_tmlp(2, 64, seed=4)
    tree = octant_tree(2)
    from paper_2604_25936_gb300 import Model
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    pts = points(n, k, seed=n + k)
    y_ref, d_ref = oracle.query(model, tree, pts, exit_layers=True)
    assert int((d_ref == 2).sum()) == k
    out = torch.full((n,), float("nan"), device="cuda")
    ws = m.workspace(n)
    m.query(torch.from_numpy(pts).cuda(), precision=prec, out=out, workspace=ws)
    torch.cuda.synchronize()
    st = m.stats(ws)
    assert st["count"][2] == k and st["count"][1] == n - k
    y = out.double().cpu().numpy()
    assert np.isfinite(y).all(), "%d rows never written" % int((~np.isfinite(y)).sum())
    err = float(np.abs(y - y_ref).max())
    assert err <= TOL[prec], (prec, n, k, err)
    m.free()
