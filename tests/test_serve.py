"""Serving loop: continuous batching over resident models (include/sand.h, sand_server_*).

The serving workload's three resident models (8 x 256 SIREN, 8 x 336 SIREN, 6 x 128 ReLU on
Fourier features, each with its own level-7 octree: synth.serve_specs) take a mix of
marching-cubes blocks and point batches from four client threads.  Every result must be
* the same in the mix as the same request run alone through sand_query_sdf (the kernels
  compute every row independently, so it is in fact expected to be bit-identical; the
  identical count is printed and required), and
* within the precision's tolerance of the FP64 oracle: 1e-5 in float32; in bf16 2e-3 for the
  sine models and, for the ReLU model (unbounded activations), twice the error of the float64
  emulation of the same bf16 operand rounding on the request's points.
Precision mixes: all bf16 (the precision the serving p99 is quoted at), all float32 on the tensor
cores (the float32 split of the 8 x 336 model reads its lo operand from shared memory) and all on
the CUDA cores.
Requests are admitted by device memory, and the latency report is consistent.
"""
import threading

import numpy as np
import pytest
import torch

import oracle
import quantised_emulation as qe
import synth

pytestmark = pytest.mark.gpu

MIXES = {"bf16": ["bf16"] * 3, "fp32": ["fp32"] * 3, "fp32_simt": ["fp32_simt"] * 3}
TOL = {"fp32": 1e-5, "fp32_simt": 1e-5, "bf16": 2e-3}


def _models():
    from paper_2604_25936_gb300 import Model
    out = []
    for model, tree in synth.serve_specs():
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
            side = int(g.choice([8, 16, 32, 40]))
            pts = synth.lattice(side)
        elif kind == 1:
            pts = g.uniform(-1, 1, (int(g.integers(1, 40000)), 3)).astype(np.float32)
        else:
            pts = g.uniform(-1.2, 1.2, (int(g.choice([1, 2, 127, 129, 4097])), 3)).astype(np.float32)
        reqs.append((int(g.integers(3)), torch.from_numpy(pts).pin_memory()))
    return reqs


@pytest.mark.parametrize("mix", sorted(MIXES))
def test_results_alone_in_the_mix_and_against_the_oracle(mix):
    from paper_2604_25936_gb300 import Server
    specs = synth.serve_specs()
    models = _models()
    precs = MIXES[mix]
    reqs = _requests(7, 48)
    alone = [models[m].query(p.cuda(), precision=precs[m]).cpu() for m, p in reqs]
    srv = Server(models, precision=precs, n_streams=3, mem_budget=256 << 20, max_batch_points=1 << 17)
    tickets = [None] * len(reqs)

    def client(idx):
        for i in idx:
            tickets[i] = srv.submit(reqs[i][0], reqs[i][1])

    threads = [threading.Thread(target=client, args=(list(range(k, len(reqs), 4)),)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    identical = [0, 0, 0]
    count = [0, 0, 0]
    worst = [0.0, 0.0, 0.0]
    for i, (m, p) in enumerate(reqs):
        out, lat = srv.wait(tickets[i])
        assert lat >= 0
        err = (out.double() - alone[i].double()).abs().max().item() if out.numel() else 0.0
        assert err <= TOL[precs[m]], "request %d (model %d, n %d): max |mix - alone| = %g" % (i, m, p.shape[0], err)
        identical[m] += int(torch.equal(out, alone[i]))
        count[m] += 1
        if not out.numel():
            continue
        model, tree = specs[m]
        pts = p.numpy()
        y_ref = oracle.query(model, tree, pts)
        e = float(np.abs(out.double().numpy() - y_ref).max())
        if precs[m] == "bf16" and model.activation == synth.ACT_RELU:
            tol = 2.0 * float(np.abs(qe.query(model, tree, pts, "bf16") - y_ref).max())
        else:
            tol = TOL[precs[m]] * max(1.0, float(np.abs(y_ref).max()))
        assert e <= tol, "request %d (model %d, %s, n %d): max |mix - oracle| = %g > %g" % (
            i, m, precs[m], p.shape[0], e, tol)
        worst[m] = max(worst[m], e)
    for k in range(3):
        print("serve %s model %d (%s): %d/%d requests identical alone and in the mix, max |err| vs oracle %.3g"
              % (mix, k, precs[k], identical[k], count[k], worst[k]))
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["points"] == sum(p.shape[0] for _, p in reqs)
    assert st["batches"] < len(reqs)  # requests were batched together
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert 0 < st["batch_ms_sum"] and 0 < st["span_ms"]
    print("serve %s: %d batches, device spans sum %.1f ms over %.1f ms of wall time (concurrency %.2f)"
          % (mix, st["batches"], st["batch_ms_sum"], st["span_ms"], st["batch_ms_sum"] / st["span_ms"]))
    srv.close()
    assert sum(identical) == len(reqs)


def test_admission_by_memory_and_errors():
    from paper_2604_25936_gb300 import SandError, Server
    models = _models()
    budget = 8 << 20  # fits about 200K points per batch
    srv = Server(models, precision=MIXES["fp32"], n_streams=3, mem_budget=budget, max_batch_points=1 << 20)
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


def test_one_handle_two_tensor_core_precisions_is_refused():
    """A model packs one tensor-core precision at a time; serving one handle in two would repack
    inside the serving loop, so the server refuses it (the CUDA-core precision needs no packing)."""
    from paper_2604_25936_gb300 import SandError, Server
    models = _models()
    with pytest.raises(SandError, match="EINVAL"):
        Server([models[0], models[0]], precision=["fp32", "bf16"])
    srv = Server([models[0], models[0]], precision=["bf16", "fp32_simt"])
    srv.close()
