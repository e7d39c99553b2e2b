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


def test_noalloc_matches_regular_query_twice():
    from paper_2604_25936_gb300 import Model, binding
    L = binding.lib()
    L.sand_query_sdf_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.POINTER(binding.QueryOpts), ctypes.c_void_p]
    L.sand_query_sdf_noalloc.restype = ctypes.c_int
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
