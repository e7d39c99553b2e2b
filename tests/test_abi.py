"""The C-ABI library loads, exports every function include/sand.h declares, agrees with
the binding's struct layouts, and rejects malformed inputs on the host — all without a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sand.h")


@pytest.fixture(scope="module")
def L():
    from paper_2604_25936_gb300 import build
    build.build()
    from paper_2604_25936_gb300 import binding
    return binding.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sand_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sand_load_tmlp", "sand_load_depth_map", "sand_query_sdf", "sand_query_sdf_grad",
                     "sand_free", "sand_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    from paper_2604_25936_gb300 import binding
    names = declared_functions()
    out = subprocess.check_output(["nm", "-D", "--defined-only", binding.LIB_PATH]).decode()
    exported = set(re.findall(r" T (sand_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(L, n)  # resolvable through ctypes
    assert set(binding.EXPORTS) <= set(names)


def test_struct_layouts_match_binding(tmp_path):
    from paper_2604_25936_gb300 import binding
    prog = tmp_path / "sizes.c"
    prog.write_text('#include "sand.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    'sizeof(sand_tmlp_desc), sizeof(sand_depth_map_desc), sizeof(sand_query_opts),'
                    'sizeof(sand_query_stats), offsetof(sand_query_opts, d_workspace), offsetof(sand_tmlp_desc, omega0),'
                    'sizeof(sand_trace_opts), offsetof(sand_trace_opts, poll_every), sizeof(sand_map_build_opts),'
                    'sizeof(sand_train_opts), offsetof(sand_train_opts, eps), sizeof(sand_server_report),'
                    'offsetof(sand_server_report, batch_ms_sum));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(binding.TmlpDesc), ctypes.sizeof(binding.DepthMapDesc), ctypes.sizeof(binding.QueryOpts),
            ctypes.sizeof(binding.QueryStats), binding.QueryOpts.d_workspace.offset, binding.TmlpDesc.omega0.offset,
            ctypes.sizeof(binding.TraceOpts), binding.TraceOpts.poll_every.offset, ctypes.sizeof(binding.MapBuildOpts),
            ctypes.sizeof(binding.TrainOpts), binding.TrainOpts.eps.offset, ctypes.sizeof(binding.ServerReport),
            binding.ServerReport.batch_ms_sum.offset]
    assert got == want


def test_host_side_validation(L, tmp_path):
    """Malformed descriptors and files fail with EFORMAT / EINVAL before any device work;
    a well-formed model on a machine without a usable device reports EUNSUPPORTED."""
    from paper_2604_25936_gb300 import binding as b
    m = synth.siren_tmlp(2, 16, seed=0)
    p = m.flat()
    h = ctypes.c_void_p()
    bad = b.TmlpDesc(0, 16, 3, 0, 0, 0, 0, 30.0)
    assert L.sand_load_tmlp_mem(ctypes.byref(bad), p.ctypes.data, p.size, 0, ctypes.byref(h)) == b.SAND_EFORMAT
    assert b"n_layers" in L.sand_last_error()
    d = b.TmlpDesc(2, 16, 3, 0, 0, 0, 0, 30.0)
    assert L.sand_load_tmlp_mem(ctypes.byref(d), p.ctypes.data, p.size - 1, 0, ctypes.byref(h)) == b.SAND_EFORMAT
    assert L.sand_load_tmlp_mem(None, p.ctypes.data, p.size, 0, ctypes.byref(h)) == b.SAND_EINVAL
    path = str(tmp_path / "m.tmlp")
    synth.save_tmlp(path, m)
    trunc = str(tmp_path / "t.tmlp")
    open(trunc, "wb").write(open(path, "rb").read()[:-8])
    assert L.sand_load_tmlp(trunc.encode(), 0, ctypes.byref(h)) == b.SAND_EFORMAT
    assert L.sand_load_tmlp(b"/nonexistent/file", 0, ctypes.byref(h)) == b.SAND_EINVAL
    rc = L.sand_load_tmlp_mem(ctypes.byref(d), p.ctypes.data, p.size, 0, ctypes.byref(h))
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        assert rc == b.SAND_EUNSUPPORTED
    else:
        assert rc == b.SAND_OK
        L.sand_free(h)
    assert L.sand_free(None) == b.SAND_OK
    st = b.QueryStats()
    assert L.sand_read_stats(None, None, ctypes.byref(st), None) == b.SAND_EINVAL
    assert L.sand_workspace_bytes(None, 1000, 0) >= 1000 * 17
    # issue-rate probes: argument errors before any device call
    sink = ctypes.c_void_p(256)
    assert L.sand_probe_rate(7, 0, 1, 1, sink, None) == b.SAND_EINVAL
    assert L.sand_probe_rate(b.PROBE_FFMA, 0, 0, 1, sink, None) == b.SAND_EINVAL
    assert L.sand_probe_rate(b.PROBE_SIN, 0, 1, 0, sink, None) == b.SAND_EINVAL
    assert L.sand_probe_rate(b.PROBE_SIN, 0, 1, 1, None, None) == b.SAND_EINVAL
    assert L.sand_probe_rate(b.PROBE_SIN, 0, 1, 1, ctypes.c_void_p(258), None) == b.SAND_EINVAL


def test_file_formats_round_trip(tmp_path):
    """The writers in synth produce the byte layout include/sand.h documents."""
    import struct
    m = synth.siren_tmlp(3, 16, seed=1, tail_kind=synth.TAIL_MULT)
    path = str(tmp_path / "m.tmlp")
    synth.save_tmlp(path, m)
    raw = open(path, "rb").read()
    assert raw[:4] == b"TMLP"
    ver, *hdr = struct.unpack("<I7i", raw[4:36])
    w0, = struct.unpack("<f", raw[36:40])
    npar, = struct.unpack("<Q", raw[40:48])
    assert ver == 1 and tuple(hdr) == m.header_ints() and w0 == np.float32(m.omega0) and npar == m.flat().size
    np.testing.assert_array_equal(np.frombuffer(raw[48:], "<f4"), m.flat())
    t = synth.voxel_sphere_octree()
    tp = str(tmp_path / "t.sdmo")
    synth.save_octree(tp, t)
    raw = open(tp, "rb").read()
    assert raw[:4] == b"SDMO"
    ver, ml, nl, nn = struct.unpack("<I3i", raw[4:20])
    assert (ver, ml, nl, nn) == (1, t.max_level, t.n_layers, t.n_nodes)
    off = 44
    np.testing.assert_array_equal(np.frombuffer(raw[off:off + 4 * nn], "<i4"), t.child)
