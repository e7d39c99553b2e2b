"""Host-side arithmetic of bench.py, without a GPU.

* flops_per_point against the per-point FLOP count of the scope table's workloads: the
  8x256 SIREN at full depth is 923,136 FLOP per point (2*3*256 + 7*2*256^2 + 8*2*256), and
  the 4x64 tiny model's SAND mix averages 5,582 FLOP per point;
* hbm_stages: 42 bytes per point (+4 per far point) over the stage time;
* the traffic record: the kernel hash ignores comments; the record's format.
"""
import os

import numpy as np

import bench


def test_flops_per_point_closed_forms():
    assert bench.flops_per_point(8, 256, False) == 2 * 3 * 256 + 7 * 2 * 256 ** 2 + 8 * 2 * 256 == 923136
    assert bench.flops_per_point(0, 256, False) == 0
    # multiplicative tails: tail 1 affine (2 W), tails 2..d two dot products (4 W)
    assert bench.flops_per_point(3, 64, True) == 2 * 3 * 64 + 2 * 2 * 64 ** 2 + 2 * 64 + 2 * 4 * 64
    # the tiny workload's histogram {1: 19456, 2: 8192, 3: 3584, 4: 1536} on the 32^3 lattice
    hist = np.array([0, 19456, 8192, 3584, 1536])
    avg = (bench.flops_per_point(np.arange(5), 64, False) * hist).sum() / hist.sum()
    assert round(avg) == 5582


def test_hbm_stages():
    r = bench.hbm_stages(1000, 10, 0.001, 6783.5)
    assert r["bytes"] == 42 * 1000 + 4 * 10
    assert abs(r["achieved"] - r["bytes"] / 1e-6 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6783.5) < 1e-12


def test_code_hash_ignores_comments(tmp_path):
    a = tmp_path / "a.cuh"
    b = tmp_path / "b.cuh"
    a.write_text("int f(int x) {  // one\n    return x + 1;\n}\n")
    b.write_text("/* header */\nint f(int x) {  // two\n\n    return x + 1;\n}\n")
    assert bench.code_sha1(str(a)) == bench.code_sha1(str(b))
    b.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.code_sha1(str(a)) != bench.code_sha1(str(b))


def test_traffic_record_format():
    """The committed record names the kernel's code hash and a per-launch byte count; bench.py
    reports it only while the hash matches the kernel source (else traffic is null)."""
    import json
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["tmlp_tc_kernel:fp32"]
    assert len(t["code_sha1"]) == 40
    assert t["dram_bytes_per_launch_full_workload"] == t["dram_bytes_read"] + t["dram_bytes_write"]
    v = bench.kernel_traffic("fp32")
    assert v is None or v == t["dram_bytes_per_launch_full_workload"]
