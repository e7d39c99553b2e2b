"""The bounded-wait abort path of the tensor-core kernel, exercised without breaking anything.

Every mbarrier wait of the kernel gives up after a limit (2 s by default).  A query may set a
much shorter limit (sand_query_opts.wait_limit_us); with 1 us the waits of an ordinary query run
out, as a hang would make them.  The kernel must then stop issuing, let its copies and MMAs
finish, free its tensor memory and return: the call completes, sand_read_stats reports
SAND_ETIMEOUT with the site that gave up, and the next query on the same model and workspace,
with the default limit, is correct again (the tensor memory was released and the flags reset).
Nothing is faulted or hung on purpose: the waits simply run out.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _query(m, x, out, ws, prec, wait_us, grad=None):
    from paper_2604_25936_gb300 import binding
    o = m._opts(prec, 0, False, None, ws)
    o.wait_limit_us = wait_us
    L = binding.lib()
    if grad is None:
        return L.sand_query_sdf(m._h, ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(out.data_ptr()),
                                ctypes.byref(o), None)
    return L.sand_query_sdf_grad(m._h, ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(grad.data_ptr()), ctypes.byref(o), None)


@pytest.mark.parametrize("prec,grad", [("fp32", False), ("bf16", False), ("fp32", True)])
def test_wait_limit_runs_out_and_the_next_query_is_correct(prec, grad):
    from paper_2604_25936_gb300 import Model, SandError, binding
    model = synth.siren_tmlp(8, 256, seed=1)
    tree = synth.scene_octree(7, 8)
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    pts = synth.lattice(64)
    x = torch.from_numpy(pts).cuda()
    n = len(pts)
    out = torch.empty(n, device="cuda")
    g = torch.empty((n, 3), device="cuda") if grad else None
    ws = m.workspace(n, grad=grad)
    for _ in range(2):  # twice in a row: the abort leaves nothing behind
        assert _query(m, x, out, ws, prec, 1, g) == binding.SAND_OK
        torch.cuda.synchronize()
        with pytest.raises(SandError, match="ETIMEOUT"):
            m.stats(ws)
    # the same query with the default limit
    assert _query(m, x, out, ws, prec, 0, g) == binding.SAND_OK
    torch.cuda.synchronize()
    st = m.stats(ws)
    assert not (st["flags"] & binding.FLAG_TIMEOUT)
    idx = synth.sample_indices(n, 4000, seed=5)
    y_ref, g_ref = oracle.query(model, tree, pts[idx], grad=True)
    tol = 1e-5 if prec == "fp32" else 2e-3
    assert np.abs(out.double().cpu().numpy()[idx] - y_ref).max() <= tol
    if grad:
        gscale = max(1.0, float(np.abs(g_ref).max()))
        assert np.abs(g.double().cpu().numpy()[idx] - g_ref).max() <= 1e-5 * model.omega0 * gscale
    m.free()


def test_wait_limit_refused_where_the_kernel_cannot_abort_safely():
    """Dynamic-exit queries synchronise their epilogue warps with a named barrier, which a partial
    abort could leave waiting, and the sphere tracer runs many queries: both refuse the option."""
    from paper_2604_25936_gb300 import Model, binding
    model = synth.siren_tmlp(2, 64, seed=3)
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    x = torch.zeros((64, 3), device="cuda")
    out = torch.empty(64, device="cuda")
    o = binding.QueryOpts()
    o.wait_limit_us = 10
    L = binding.lib()
    rc = L.sand_query_sdf_dynamic(m._h, ctypes.c_void_p(x.data_ptr()), 64, ctypes.c_float(0.01),
                                  ctypes.c_void_p(out.data_ptr()), None, ctypes.byref(o), None)
    assert rc == binding.SAND_EINVAL
    m.free()
