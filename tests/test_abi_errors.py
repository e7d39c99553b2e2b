"""Argument errors at the C-ABI boundary, without a GPU.

Every entry point that takes a model, a server or a buffer must refuse a NULL handle or a
malformed argument with SAND_EINVAL and a message (sand_last_error), before any device
work, and the calls documented as no-ops on NULL must return SAND_OK.
"""
import ctypes

import pytest


@pytest.fixture(scope="module")
def B():
    from paper_2604_25936_gb300 import binding, build
    build.build()
    L = binding.lib()
    L.sand_query_sdf_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
    L.sand_query_sdf_noalloc.restype = ctypes.c_int
    return binding


def _einval(B, rc):
    assert rc == B.SAND_EINVAL, rc
    assert len(B.lib().sand_last_error()) > 0


def test_null_model_is_refused_everywhere(B):
    L = B.lib()
    P = ctypes.c_void_p
    buf = P(256)  # never dereferenced: the NULL model is refused first
    o = B.QueryOpts()
    _einval(B, L.sand_query_sdf(None, buf, 10, buf, ctypes.byref(o), None))
    _einval(B, L.sand_query_sdf_grad(None, buf, 10, buf, buf, ctypes.byref(o), None))
    _einval(B, L.sand_query_sdf_host(None, buf, 10, buf, ctypes.byref(o), None))
    _einval(B, L.sand_query_sdf_noalloc(None, buf, 10, buf, ctypes.byref(o), None))
    _einval(B, L.sand_query_sdf_dynamic(None, buf, 10, ctypes.c_float(0.01), buf, None, ctypes.byref(o), None))
    d = B.TmlpDesc()
    _einval(B, L.sand_model_desc(None, ctypes.byref(d)))
    _einval(B, L.sand_load_depth_map(None, b"x.sdmo"))
    dm = B.DepthMapDesc()
    _einval(B, L.sand_load_depth_map_mem(None, ctypes.byref(dm), buf, buf, None))
    st = B.QueryStats()
    _einval(B, L.sand_read_stats(None, buf, ctypes.byref(st), None))
    tr = B.TraceOpts(8, 1e-4, 8, 0)
    _einval(B, L.sand_sphere_trace(None, buf, 0, buf, 10, ctypes.byref(tr), ctypes.byref(o), buf, buf, buf, None, None))
    mb = B.MapBuildOpts(4, 1.5e-4, 0, 0)
    _einval(B, L.sand_build_depth_map(None, ctypes.byref(dm), buf, buf, ctypes.byref(mb), buf, None))
    assert L.sand_free(None) == B.SAND_OK


def test_server_handles(B):
    L = B.lib()
    h = ctypes.c_void_p()
    _einval(B, L.sand_server_create(None, 1, None, ctypes.byref(h)))
    models = (ctypes.c_void_p * 2)(None, None)
    _einval(B, L.sand_server_create(models, 2, None, ctypes.byref(h)))  # NULL model in the list
    _einval(B, L.sand_server_create(models, 0, None, ctypes.byref(h)))
    t = ctypes.c_uint64()
    _einval(B, L.sand_server_submit(None, 0, None, 0, None, ctypes.byref(t)))
    _einval(B, L.sand_server_wait(None, 1, 1.0, None))
    rep = B.ServerReport()
    _einval(B, L.sand_server_stats(None, ctypes.byref(rep)))
    assert L.sand_server_destroy(None) == B.SAND_OK


def test_trainer_entry_points_refuse_null(B):
    L = B.lib()
    P = ctypes.c_void_p
    h = P()
    buf = P(256)
    _einval(B, L.sand_trainer_create(None, None, ctypes.byref(h)))
    _einval(B, L.sand_train_step(None, buf, buf, 10, None, None, 1, None))
    _einval(B, L.sand_trainer_params(None, buf, 10))
    _einval(B, L.sand_trainer_commit(None))
    _einval(B, L.sand_trainer_status(None, None))
    assert L.sand_trainer_destroy(None) == B.SAND_OK


def test_sizes_without_a_device(B):
    L = B.lib()
    # workspace: a 1 KiB header, per-block histograms, then 17 B per point (exit byte, float4 row)
    w0 = L.sand_workspace_bytes(None, 0, 0)
    w1 = L.sand_workspace_bytes(None, 1 << 20, 0)
    assert w1 - w0 >= 17 * (1 << 20)
    assert L.sand_workspace_bytes(None, 1 << 20, 1) == w1  # the gradient needs no more
    # tracer state: grows with the rays, about 60 B per ray
    s1, s2 = L.sand_trace_state_bytes(1 << 16), L.sand_trace_state_bytes(1 << 17)
    assert 40 * (1 << 16) <= s2 - s1 <= 200 * (1 << 16)


def test_model_file_fuzz(B, tmp_path):
    """Truncations and single-byte corruptions of a model file give a status, never a crash
    or an allocation sized by a corrupted count: EFORMAT for a broken header, size or
    descriptor; a well-formed file parses (EUNSUPPORTED without a usable device, else OK)."""
    import numpy as np
    import synth
    L = B.lib()
    m = synth.siren_tmlp(2, 16, seed=3)
    path = tmp_path / "m.tmlp"
    synth.save_tmlp(str(path), m)
    raw = path.read_bytes()
    try:
        import torch
        good = B.SAND_OK if torch.cuda.is_available() else B.SAND_EUNSUPPORTED
    except Exception:
        good = B.SAND_EUNSUPPORTED
    allowed = {B.SAND_EFORMAT, B.SAND_EINVAL, good}
    h = ctypes.c_void_p()
    g = np.random.Generator(np.random.PCG64(1))
    cases = [raw[:k] for k in (0, 3, 4, 8, 20, 40, 47, 48, 52, len(raw) - 1)]
    for _ in range(200):
        b = bytearray(raw)
        i = int(g.integers(0, 48))  # the header: magic, version, 7 ints, omega0, parameter count
        b[i] = int(g.integers(0, 256))
        cases.append(bytes(b))
    # the parameter count set to the largest value the header accepts (2^31 - 1)
    b = bytearray(raw)
    b[40:48] = (2 ** 31 - 1).to_bytes(8, "little")
    cases.append(bytes(b))
    for k, data in enumerate(cases):
        f = tmp_path / ("c%d.tmlp" % k)
        f.write_bytes(data)
        rc = L.sand_load_tmlp(str(f).encode(), 0, ctypes.byref(h))
        assert rc in allowed, (k, rc, L.sand_last_error())
        if rc == B.SAND_OK:
            L.sand_free(h)
    big = tmp_path / "big.tmlp"
    big.write_bytes(cases[-1])
    assert L.sand_load_tmlp(str(big).encode(), 0, ctypes.byref(h)) == B.SAND_EFORMAT
