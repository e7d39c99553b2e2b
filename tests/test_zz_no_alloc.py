"""sand_query_sdf_noalloc: the SAND query for callers that must not allocate device memory.

Such callers (a framework whose memory pool owns the GPU budget, a latency-critical
serving loop that cannot take cudaMalloc's implicit synchronisation) get their
query scratch from a static device array inside libsand.  This file is named to be
collected last.  It calls the entry point through the C-ABI twice in a row and
checks each result against the regular sand_query_sdf within the float32
tolerance (1e-5), and checks the size limit.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2604_25936_gb300 import binding
    L = binding.lib()
    L.sand_query_sdf_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.POINTER(binding.QueryOpts), ctypes.c_void_p]
    L.sand_query_sdf_noalloc.restype = ctypes.c_int
    return L


def test_noalloc_matches_regular_query_twice():
    from paper_2604_25936_gb300 import Model, binding
    L = _lib()
    model = synth.siren_tmlp(8, 256, seed=1)
    tree = synth.scene_octree(7, 8)
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    stream = torch.cuda.current_stream()
    inputs = [synth.lattice(64), synth.uniform_points(300001, seed=44)]
    for prec in ("fp32_simt", "fp32"):
        for call, pts in enumerate(inputs):
            x = torch.from_numpy(pts).cuda()
            ref = m.query(x, precision=prec)  # regular entry point (also packs this precision's weights)
            out = torch.full((len(pts),), float("nan"), device="cuda")
            o = binding.QueryOpts()
            o.precision = binding.PRECISION[prec]
            rc = L.sand_query_sdf_noalloc(m._h, ctypes.c_void_p(x.data_ptr()), len(pts), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream))
            assert rc == binding.SAND_OK, L.sand_last_error()
            torch.cuda.synchronize()
            err = (out.double() - ref.double()).abs().max().item()
            assert err <= 1e-5, "call %d (%s): max |noalloc - regular| = %g" % (call, prec, err)
    # sizes beyond the static scratch are refused with a clear error
    big = torch.zeros((2 ** 20 + 1, 3), device="cuda")
    outb = torch.empty(2 ** 20 + 1, device="cuda")
    rc = L.sand_query_sdf_noalloc(m._h, ctypes.c_void_p(big.data_ptr()), big.shape[0], ctypes.c_void_p(outb.data_ptr()),
                                  None, ctypes.c_void_p(stream.cuda_stream))
    assert rc == binding.SAND_EINVAL and b"no-allocation scratch" in L.sand_last_error()
    m.free()


def test_noalloc_first_call_allocates_nothing():
    """On a fresh model, with the CUDA-core precision (whose weights exist from loading), the
    no-allocation entry point runs before any regular query: the model's own workspace is
    never created (sand_read_stats without a workspace still finds none), the device's free
    memory is the same before and after a later call (the first call looks up the scratch
    array, and with lazy module loading that also loads the library's module and its kernels
    on this device), and every result matches the regular query run afterwards."""
    from paper_2604_25936_gb300 import Model, binding
    L = _lib()
    model = synth.siren_tmlp(4, 64, seed=0)
    tree = synth.voxel_sphere_octree()
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    pts = synth.lattice(32)
    x = torch.from_numpy(pts).cuda()
    stream = torch.cuda.current_stream()
    o = binding.QueryOpts()
    o.precision = binding.PRECISION["fp32_simt"]
    outs = [torch.full((len(pts),), float("nan"), device="cuda") for _ in range(3)]
    free = []
    for out in outs:
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        rc = L.sand_query_sdf_noalloc(m._h, ctypes.c_void_p(x.data_ptr()), len(pts), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream))
        assert rc == binding.SAND_OK, L.sand_last_error()
        torch.cuda.synchronize()
    assert free[1] == free[2]
    st = binding.QueryStats()
    rc = L.sand_read_stats(m._h, None, ctypes.byref(st), ctypes.c_void_p(stream.cuda_stream))
    assert rc == binding.SAND_EINVAL and b"no workspace" in L.sand_last_error()
    ref = m.query(x, precision="fp32_simt")
    for out in outs:
        assert (out.double() - ref.double()).abs().max().item() <= 1e-5
    m.free()


def test_noalloc_unsupported_precision_says_so():
    """A precision the model cannot take at all (FP8 on a ReLU network) is refused as
    unsupported, not as 'query once first'."""
    from paper_2604_25936_gb300 import Model, binding
    L = _lib()
    model = synth.relu_ff_tmlp(3, 64, n_freq=32, sigma=4.0, seed=3)
    m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    tree = synth.voxel_sphere_octree()
    m.set_depth_map(tree.max_level, 3, tree.child, np.minimum(tree.depth, 3), tree.far)
    x = torch.zeros((10, 3), device="cuda")
    out = torch.empty(10, device="cuda")
    o = binding.QueryOpts()
    o.precision = binding.PRECISION["fp8"]
    rc = L.sand_query_sdf_noalloc(m._h, ctypes.c_void_p(x.data_ptr()), 10, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.byref(o), None)
    assert rc == binding.SAND_EUNSUPPORTED and b"not supported" in L.sand_last_error()
    m.free()
