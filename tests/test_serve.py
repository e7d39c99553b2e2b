"""Serving loop: continuous batching over resident models (include/sand.h, sand_server_*).

Results must be the same alone and in the mix (float32 tolerance 1e-5; the
kernels compute every row independently, so they are in fact expected to be
bit-identical), requests are admitted by device memory, and the latency report
is consistent.
"""
import threading

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _models():
    from paper_2604_25936_gb300 import Model
    specs = [(synth.siren_tmlp(8, 256, seed=1), synth.scene_octree(7, 8)),
             (synth.relu_ff_tmlp(6, 128, n_freq=64, sigma=10.0, seed=3), synth.scene_octree(7, 6, transform=synth.rotation([1, 1, 0], 0.7), scale=0.9)),
             (synth.siren_tmlp(4, 64, seed=0), synth.voxel_sphere_octree())]
    out = []
    for model, tree in specs:
        m = Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
        out.append(m)
    return out


def _requests(seed, count):
    g = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(count):
        kind = g.integers(3)
        if kind == 0:
            side = int(g.choice([8, 16, 32, 48]))
            pts = synth.lattice(side)
        elif kind == 1:
            pts = g.uniform(-1, 1, (int(g.integers(1, 70000)), 3)).astype(np.float32)
        else:
            pts = g.uniform(-1.2, 1.2, (int(g.choice([1, 2, 127, 129, 4097])), 3)).astype(np.float32)
        reqs.append((int(g.integers(3)), torch.from_numpy(pts).pin_memory()))
    return reqs


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_results_alone_and_in_the_mix(precision):
    from paper_2604_25936_gb300 import Server
    models = _models()
    reqs = _requests(7, 60)
    alone = [models[m].query(p.cuda(), precision=precision).cpu() for m, p in reqs]
    srv = Server(models, precision=precision, n_streams=3, mem_budget=256 << 20, max_batch_points=1 << 17)
    tickets = [None] * len(reqs)

    def client(idx):
        for i in idx:
            tickets[i] = srv.submit(reqs[i][0], reqs[i][1])

    threads = [threading.Thread(target=client, args=(list(range(k, len(reqs), 4)),)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    identical = 0
    for i, (m, p) in enumerate(reqs):
        out, lat = srv.wait(tickets[i])
        assert lat >= 0
        err = (out.double() - alone[i].double()).abs().max().item() if out.numel() else 0.0
        assert err <= 1e-5, "request %d (model %d, n %d): max |mix - alone| = %g" % (i, m, p.shape[0], err)
        identical += int(torch.equal(out, alone[i]))
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["points"] == sum(p.shape[0] for _, p in reqs)
    assert st["batches"] < len(reqs)  # requests were batched together
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()
    assert identical == len(reqs)


def test_admission_by_memory_and_errors():
    from paper_2604_25936_gb300 import SandError, Server
    models = _models()
    from paper_2604_25936_gb300 import binding
    budget = 8 << 20  # fits about 200K points per batch
    srv = Server(models, precision="fp32", n_streams=3, mem_budget=budget, max_batch_points=1 << 20)
    g = np.random.Generator(np.random.PCG64(11))
    reqs = [g.uniform(-1, 1, (100000, 3)).astype(np.float32) for _ in range(12)]
    tickets = [srv.submit(0, p) for p in reqs]
    outs = [srv.wait(t)[0] for t in tickets]
    for p, o in zip(reqs, outs):
        ref = models[0].query(torch.from_numpy(p).cuda(), precision="fp32").cpu().numpy()
        assert np.abs(o.astype(np.float64) - ref).max() <= 1e-5
    big = srv.submit(0, np.zeros((2_000_000, 3), np.float32))  # can never fit the arena
    with pytest.raises(SandError, match="ENOMEM"):
        srv.wait(big)
    empty = srv.submit(1, np.zeros((0, 3), np.float32))
    assert srv.wait(empty)[0].size == 0
    with pytest.raises(SandError, match="EINVAL"):
        srv.submit(5, reqs[0])
    srv.close()
