"""Benchmark of the SAND query path on GB300.

One step = one SAND query over a 256^3 marching-cubes lattice (16,777,216
points): depth-map lookup, exit-layer binning and the T-MLP to each point's
exit layer, for an 8 x 256 SIREN T-MLP (random SIREN init, seed 1, linear
tails) and a level-7 octree built from an analytic scene.  The same T-MLP run
to full depth on the same points is timed beside it.  Inputs are larger than
L2 (201 MB of points), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank evaluates its own
full lattice (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

GRID = 256
N_LAYERS, WIDTH, SEED = 8, 256, 1
TOL = {"fp32": 1e-5, "fp32_simt": 1e-5, "fp16": 2e-3, "bf16": 2e-3, "fp8": None}
DTYPE = {"fp32": "f32 (3 x f16 split, f32 accumulate)", "fp32_simt": "f32", "fp16": "f16 (f32 accumulate)",
         "bf16": "bf16 (f32 accumulate)", "fp8": "e4m3 (f32 accumulate)"}
KERNEL_SRC = {"fp32_simt": "paper_2604_25936_gb300/csrc/tmlp_simt.cu", "fp32": "paper_2604_25936_gb300/csrc/tc_kernel.cuh",
              "fp16": "paper_2604_25936_gb300/csrc/tc_kernel.cuh", "bf16": "paper_2604_25936_gb300/csrc/tc_kernel.cuh",
              "fp8": "paper_2604_25936_gb300/csrc/tc_kernel.cuh"}
KERNEL_NAME = {"fp32_simt": "tmlp_simt_kernel", "fp32": "tmlp_tc_kernel", "fp16": "tmlp_tc_kernel",
               "bf16": "tmlp_tc_kernel", "fp8": "tmlp_tc_kernel"}
METRIC = "SDF queries/s, SAND vs full-depth T-MLP on 1 GB300 at stated error; serve p99 ms"
WORKLOAD = "SAND-SIREN 8x256 linear tails, level-7 octree, %d^3 lattice" % GRID


def hbm_stages(n: int, n_far: int, ms: float, peak_gbs: float) -> dict:
    """Bandwidth of the memory-bound stages of a SAND query (workspace reset, lookup, scan,
    scatter): the lookup reads a point (12 B) and writes its exit layer (1 B; far points also
    their stored value, 4 B); the scatter reads both again (13 B) and writes the sorted row
    (16 B); the per-block histograms are a few KB."""
    bytes_ = 42 * n + 4 * n_far
    gbs = bytes_ / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    return {"kernels": "lookup_kernel + scan_kernel + scatter_kernel", "bytes_per_point": 42,
            "bytes": bytes_, "ms": ms, "achieved": gbs, "peak": peak_gbs, "unit": "GB/s",
            "frac": gbs / peak_gbs if peak_gbs else None}


def flops_per_point(d: np.ndarray, W: int, tail_mult: bool) -> np.ndarray:
    """Algorithmic FLOPs of a point that exits at layer d >= 1: layer 1 (2*3*W),
    d-1 hidden products (2*W^2 each) and d tails (2*W, or 4*W for multiplicative tails >= 2)."""
    d = np.asarray(d, np.float64)
    tails = d * 2 * W if not tail_mult else (2 * W + (d - 1) * 4 * W)
    return np.where(d >= 1, 2 * 3 * W + (d - 1) * 2 * W * W + tails, 0.0)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while the timed region runs."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[0]]
            rows = mine or rows
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [v for v in sm if mx and v >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def code_sha1(path: str) -> str:
    """sha1 of a C/CUDA source with its comments and blank lines removed: a change to the
    comments alone leaves the kernel, and so the counters taken from it, unchanged."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
    return hashlib.sha1("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()


def kernel_traffic(prec: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    when the kernel's code changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        t = json.load(open(path)).get(KERNEL_NAME[prec] + ":" + prec)
        if t and t.get("code_sha1") == code_sha1(os.path.join(ROOT, KERNEL_SRC[prec])):
            return t.get("dram_bytes_per_launch_full_workload")
    except Exception:
        return None
    return None


def host_cpu() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm implementer and part)."""
    try:
        fields = {}
        for ln in open("/proc/cpuinfo"):
            k, _, v = ln.partition(":")
            fields.setdefault(k.strip(), v.strip())
        if fields.get("model name"):
            return fields["model name"]
        if fields.get("CPU implementer"):
            return "Arm implementer %s part %s" % (fields.get("CPU implementer"), fields.get("CPU part", "?"))
    except OSError:
        pass
    return "unknown"


def cpu_baseline(model, tree, pts, budget_s: float = 12.0):
    """The FP64 oracle as it stands, on the host cores, over a seeded sample of the lattice."""
    import oracle
    n = len(pts)
    probe = synth.sample_indices(n, 20000, seed=11)
    t0 = time.perf_counter()
    oracle.query(model, tree, pts[probe])
    rate = 20000 / max(time.perf_counter() - t0, 1e-6)
    k = int(min(n, max(20000, rate * budget_s)))
    idx = synth.sample_indices(n, k, seed=11)
    t0 = time.perf_counter()
    oracle.query(model, tree, pts[idx])
    dt = time.perf_counter() - t0
    # the oracle's own full-depth mode on 20,000 lattice points (PCG64 seed 12), for its SAND / full ratio
    kf = min(n, 20000)
    idf = synth.sample_indices(n, kf, seed=12)
    t0 = time.perf_counter()
    oracle.full_depth(model, pts[idf])
    dtf = time.perf_counter() - t0
    return {"value": k / dt, "unit": "queries/s", "cores": oracle.threads(), "kind": "oracle",
            "nproc": os.cpu_count(), "cpu": host_cpu(),
            "full_depth_value": kf / dtf, "full_depth_sample": "%d lattice points (PCG64 seed 12), %.1f s" % (kf, dtf),
            "sample": "%d lattice points drawn with PCG64 seed 11 from the %d^3 lattice, SAND query (lookup + "
                      "T-MLP to each exit layer) in float64, %.1f s" % (k, GRID, dt)}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload, a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED)
    tree = synth.scene_octree(7, N_LAYERS)
    pts = synth.lattice(GRID)
    probe = synth.sample_indices(len(pts), 10000, seed=11)
    t0 = time.perf_counter()
    oracle.query(model, tree, pts[probe])
    rate = 10000 / max(time.perf_counter() - t0, 1e-6)
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    k = int(min(len(pts), max(10000, rate * per_step)))
    idx = synth.sample_indices(len(pts), k, seed=11)
    sample = pts[idx]
    for _ in range(args.warmup):
        oracle.query(model, tree, sample)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.query(model, tree, sample)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = k / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": len(pts), "sample_per_step": k},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": oracle.threads(), "kind": "oracle",
                             "nproc": os.cpu_count(), "cpu": host_cpu(),
                             "sample": "%d lattice points (PCG64 seed 11) per step, float64 SAND query" % k},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(seconds: float, world: int, device=None) -> float:
    """Maximum of a per-rank duration over all ranks (the job ends when the slowest rank does)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job queries/s under weak scaling: every rank evaluates its own points_per_rank."""
    return world * points_per_rank / max_seconds


def serve_models(sand):
    """The three resident models of the serving workload, each with its own level-7 octree."""
    models = []
    for model, tree in synth.serve_specs():
        m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
        models.append(m)
    return models


def serve_requests(count: int, seed: int):
    """Request pool: half marching-cubes blocks (side 32/64/128/256 with equal probability, a
    side^3 lattice over a random sub-cube), half ray-sample batches (n log-uniform in
    [4096, 2^21], points along random rays through the domain); model uniform over 3."""
    import torch
    g = np.random.Generator(np.random.PCG64(seed))
    pool = []
    for _ in range(count):
        if g.random() < 0.5:
            side = int(g.choice([32, 64, 128, 256]))
            ext = g.uniform(0.25, 2.0)
            lo = g.uniform(-1.0, 1.0 - ext, 3)
            t = np.arange(side, dtype=np.float64) / max(side - 1, 1) * ext
            z, y, x = np.meshgrid(t + lo[2], t + lo[1], t + lo[0], indexing="ij")
            pts = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32)
        else:
            n = int(np.exp(g.uniform(np.log(4096), np.log(1 << 21))))
            o = g.uniform(-1, 1, (n, 3)); d = g.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
            pts = np.clip(o + d * g.uniform(0, 0.5, (n, 1)), -1.2, 1.2).astype(np.float32)
        pool.append((int(g.integers(3)), torch.from_numpy(pts).pin_memory()))
    return pool


def _open_loop(sand, srv, pool, lam: float, seconds: float, g):
    """Poisson arrivals at lam requests/s for `seconds`, each a uniformly drawn pool entry with
    an output buffer of its own (buffers are recycled once their request completed, and a new
    pinned buffer is made when none is free), so no arrival is ever dropped.  Returns the
    server's report plus the arrivals submitted and the most requests outstanding at once."""
    import collections
    import threading
    import torch
    free_out = [[] for _ in pool]
    pending = collections.deque()
    lock = threading.Lock()
    done = threading.Event()
    outstanding = [0, 0]

    def waiter():
        while True:
            with lock:
                item = pending.popleft() if pending else None
            if item is None:
                if done.is_set():
                    return
                time.sleep(0.0002)
                continue
            t, i, buf = item
            srv.wait(t)
            with lock:
                free_out[i].append(buf)
                outstanding[0] -= 1

    th = threading.Thread(target=waiter)
    th.start()
    t_end = time.perf_counter() + seconds
    nxt = time.perf_counter()
    sent = 0
    while True:
        nxt += g.exponential(1.0 / lam)
        if nxt >= t_end:
            break
        while time.perf_counter() < nxt:
            time.sleep(max(0.0, min(0.002, nxt - time.perf_counter())))
        i = int(g.integers(len(pool)))
        with lock:
            buf = free_out[i].pop() if free_out[i] else None
        if buf is None:
            buf = torch.empty(pool[i][1].shape[0], dtype=torch.float32).pin_memory()
        t = srv.submit(pool[i][0], pool[i][1], buf)
        with lock:
            pending.append((t, i, buf))
            outstanding[0] += 1
            outstanding[1] = max(outstanding[1], outstanding[0])
        sent += 1
    done.set()
    th.join()
    st = srv.stats()
    st.update({"offered_requests_per_s": lam, "submitted": sent, "dropped": 0, "max_outstanding": outstanding[1],
               "seconds": seconds})
    return st


def serve_bench(sand, models, precision, pool, run_s: float, sweep_s: float, mem_budget: int = 16 << 30):
    """Continuous batching over the three resident models: a closed burst of the pool estimates
    the saturation rate; open-loop Poisson runs of sweep_s seconds at 0.25 .. 1.5 of that
    estimate, and beyond while the server keeps up, find the saturation throughput (the largest
    completed queries/s); then open-loop
    runs of run_s seconds at 0.5x and 0.8x of saturation report p50 / p99 request latency
    (submit to result) and aggregate queries/s."""
    import torch
    precs = {"bf16": ["bf16", "bf16", "bf16"], "fp32": ["fp32", "fp32", "fp32"]}[precision]
    out = {"precision_per_model": precs, "n_streams": 4, "mem_budget": mem_budget}

    def server():
        return sand.Server(models, precision=precs, n_streams=4, mem_budget=mem_budget, max_batch_points=1 << 22)

    outs = [torch.empty(p.shape[0], dtype=torch.float32).pin_memory() for _, p in pool]
    srv = server()
    for i in range(min(4, len(pool))):  # warm up
        srv.wait(srv.submit(pool[i][0], pool[i][1], outs[i]))
    srv.close()
    srv = server()
    t0 = time.perf_counter()
    tk = [srv.submit(m, p, outs[i]) for i, (m, p) in enumerate(pool)]
    for t in tk:
        srv.wait(t)
    burst_s = time.perf_counter() - t0
    srv.close()
    pts_total = sum(p.shape[0] for _, p in pool)
    mean_pts = pts_total / len(pool)
    burst_qps = pts_total / burst_s
    out["burst_qps"] = burst_qps
    g = np.random.Generator(np.random.PCG64(99))
    sweep = []
    # 0.25 .. 1.5 of the burst estimate, then on in steps of 0.5 (up to 4) while the server still
    # keeps up (completes at least 95 % of the offered rate): a short burst can under-read the
    # saturation rate, and the load levels below are fractions of the largest completed rate
    fracs = [0.25, 0.5, 0.75, 1.0, 1.25, 1.5]
    i = 0
    while i < len(fracs):
        frac = fracs[i]
        srv = server()
        st = _open_loop(sand, srv, pool, frac * burst_qps / mean_pts, sweep_s, g)
        srv.close()
        sweep.append({"offered_fraction_of_burst": frac, "offered_queries_per_s": frac * burst_qps,
                      "queries_per_s": st["queries_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                      "requests": st["requests"], "max_outstanding": st["max_outstanding"]})
        if i == len(fracs) - 1 and st["queries_per_s"] >= 0.95 * frac * burst_qps and frac < 4.0:
            fracs.append(frac + 0.5)
        i += 1
    sat_qps = max(e["queries_per_s"] for e in sweep)
    out["lambda_sweep"] = sweep
    out["saturation_qps"] = sat_qps
    for frac in (0.5, 0.8):
        srv = server()
        st = _open_loop(sand, srv, pool, frac * sat_qps / mean_pts, run_s, g)
        srv.close()
        out["load_%.1f" % frac] = {k: st[k] for k in ("offered_requests_per_s", "submitted", "dropped", "requests",
                                                      "batches", "p50_ms", "p99_ms", "max_ms", "queries_per_s",
                                                      "max_outstanding", "seconds")}
        # batches in flight at once on the device: sum of per-batch device spans / wall span
        out["load_%.1f" % frac]["device_concurrency"] = st["batch_ms_sum"] / st["span_ms"] if st["span_ms"] else None
    return out


def train_bench(sand, local: int, steps: int, n: int = 100000):
    """Training steps of the benchmark's 8 x 256 SIREN T-MLP (Sec. 3.3: the loss of Eq. 4 / Eq. 8
    over every tail, its gradient, one Adam update) on a batch of n points sampled as Sec. 4.1
    describes (60 % on the analytic scene's surface, 40 % moved by Gaussian noise of sigma 0.01)
    with their exact SDF as targets.  Algorithmic work per step: the forward pass
    (2*3*W + (L-1)*2*W^2 + L*2*W per point), the backward products W_l^T delta_l and the weight
    gradients delta_l h_{l-1}^T ((L-1)*2*W^2 each per point, plus 2*3*W for W_1)."""
    import torch
    from paper_2604_25936_gb300.binding import Trainer
    model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED)
    pts, gt = synth.training_batch(n, seed=21)
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    tr = Trainer(m, max_points=n)
    x, t = torch.from_numpy(pts).cuda(), torch.from_numpy(gt).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    for _ in range(3):
        tr.step(x, t, loss=loss)
    torch.cuda.synchronize()
    first = float(loss.item())
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        tr.step(x, t, loss=loss)
    t1.record(stream)
    torch.cuda.synchronize()
    tr.status()
    ms = t0.elapsed_time(t1) / steps
    L, W = N_LAYERS, WIDTH
    fwd = 2 * 3 * W + (L - 1) * 2 * W * W + L * 2 * W
    flops = float(n) * (fwd + 2 * (L - 1) * 2 * W * W + 2 * 3 * W)
    pk, pk_src = peaks()
    peak = pk.get("bf16_tflops_sustained", 1700.0) / 3.0
    achieved = flops / (ms / 1e3) / 1e12
    out = {"model": "8x256 SIREN, linear tails", "batch_points": n, "sampling": "60% surface, 40% surface + N(0, 0.01^2)",
           "ms_per_step": ms, "steps_per_s": 1e3 / ms, "points_per_s": n / (ms / 1e3),
           "loss_after_warmup": first, "loss_after_timed": float(loss.item()),
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "peak_source": "%s bf16 sustained / 3 (float32 split products)" % pk_src},
           "paper_context": "Table 9: 0.0241 s per T-MLP training iteration (SIREN 8x256, RTX 4090, PyTorch, batch not stated)"}
    tr.close()
    m.free()
    return out


def deep_map_bench(sand, local: int, steps: int, level: int = 9):
    """The benchmark lattice query (8 x 256 SIREN, float32 mode) against the analytic scene's octree
    refined to `level` (the paper's octrees go to depth 9-10, Table 5), which the library keeps
    in its brick encoding: SAND queries/s and the bandwidth of the memory-bound stages (lookup,
    scan, scatter: 42 B per network point) against the HBM copy rate."""
    import torch
    model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED)
    tree = synth.scene_octree(level, N_LAYERS)
    pts = synth.lattice(GRID)
    n = len(pts)
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    x = torch.from_numpy(pts).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ws = m.workspace(n)
    for _ in range(3):
        m.query(x, precision="fp32", out=out, workspace=ws)
    torch.cuda.synchronize()
    counts = np.array(m.stats(ws)["count"][:N_LAYERS + 1], np.int64)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        m.query(x, precision="fp32", out=out, workspace=ws, events=ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    step_ms = t0.elapsed_time(t1) / steps
    pre_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    pk, _ = peaks()
    m.free()
    return {"octree_level": level, "octree_nodes": int(tree.n_nodes), "encoding": "bricks of 8^3 finest cells",
            "queries_per_s": n / (step_ms / 1e3), "ms_per_step": step_ms,
            "exit_layer_histogram": {str(d): int(c) for d, c in enumerate(counts)},
            "hbm_stages": hbm_stages(n, int(counts[0]), pre_ms, pk.get("hbm_gbs", 6800.0))}


def paper_variants(sand, local: int, steps: int, prec: str, peak_tflops: float, hbm_gbs: float):
    """The benchmark lattice query as the paper states the method: (a) multiplicative tails for
    layers >= 2 (Eq. 3), and (b) the far-field depth map, whose leaves away from the surface
    hold exit layer 0 and answer with the SDF stored at their centre (Eq. 7).  Each: SAND
    queries/s, the T-MLP kernel's algorithmic TFLOP/s against the precision's peak, the error
    against the oracle on 20,000 sampled lattice points; (b) also the whole step's algorithmic
    traffic (12 B read + 4 B written per point) against the HBM copy rate."""
    import torch
    import oracle
    pts = synth.lattice(GRID)
    n = len(pts)
    x = torch.from_numpy(pts).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    idx = synth.sample_indices(n, 20000, seed=11)
    res = {"lattice": "%d^3 (%d points)" % (GRID, n), "precision": prec}
    for name, tail, far in (("mult_tails", synth.TAIL_MULT, False), ("far_field", synth.TAIL_LINEAR, True)):
        model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED, tail_kind=tail)
        tree = synth.scene_octree(7, N_LAYERS, far_field=far)
        m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
        ws = m.workspace(n)
        for _ in range(3):
            m.query(x, precision=prec, out=out, workspace=ws)
        torch.cuda.synchronize()
        counts = np.array(m.stats(ws)["count"][:N_LAYERS + 1], np.int64)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(steps):
            m.query(x, precision=prec, out=out, workspace=ws, events=ev[k])
        t1.record(stream)
        torch.cuda.synchronize()
        step_ms = t0.elapsed_time(t1) / steps
        mlp_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / steps
        pre_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
        flops = float((flops_per_point(np.arange(N_LAYERS + 1), WIDTH, tail == synth.TAIL_MULT) * counts).sum())
        achieved = flops / (mlp_ms / 1e3) / 1e12
        y_ref = oracle.query(model, tree, pts[idx])
        entry = {"queries_per_s": n / (step_ms / 1e3), "ms_per_step": step_ms, "tmlp_ms": mlp_ms,
                 "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                              "frac": achieved / peak_tflops, "kernel": KERNEL_NAME[prec]},
                 "max_abs_err_vs_oracle_20k": float(np.abs(out.cpu().numpy()[idx].astype(np.float64) - y_ref).max()),
                 "exit_layer_histogram": {str(d): int(c) for d, c in enumerate(counts)}}
        if far:
            # the memory-bound stages: the lookup reads a point and writes its exit byte (far points
            # also their stored value); the scatter reads every exit byte and copies the network
            # points into sorted 16-byte rows
            n_far = int(counts[0])
            n_net = n - n_far
            bytes_ = 14.0 * n + 4.0 * n_far + 28.0 * n_net
            gbs = bytes_ / (pre_ms / 1e3) / 1e9
            entry["far_points"] = n_far
            entry["lookup_bin_ms"] = pre_ms
            entry["hbm"] = {"kernels": "lookup_kernel + scan_kernel + scatter_kernel", "bytes": bytes_,
                            "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                            "algorithmic_bytes_per_point": 16,
                            "step_achieved_of_algorithmic": 16.0 * n / (step_ms / 1e3) / 1e9}
        res[name] = entry
        m.free()
    return res


def precision_variant(sand, local: int, steps: int, grid: int = 512, n_err: int = 1 << 20, sine_rate: float = 0.0):
    """8 x 256 and 8 x 336 SAND-SIRENs on a grid^3 lattice with bf16 and FP8 hidden products (and
    the 8 x 336 one in the float32 split too): SAND and full-depth queries/s, tensor-core TFLOP/s,
    the sine pipe's share, and the error against the FP64 oracle on n_err uniform points in
    [-1, 1]^3 (PCG64 seed 7; full depth on the first 20,000)."""
    import torch
    import oracle
    pts = synth.lattice(grid)
    n = len(pts)
    x = torch.from_numpy(pts).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    upts = synth.uniform_points(n_err, seed=7)
    ux = torch.from_numpy(upts).cuda()
    stream = torch.cuda.current_stream()
    res = {"lattice": "%d^3 (%d points)" % (grid, n), "error_sample": "%d uniform points, PCG64 seed 7" % n_err}
    for width, seed, tree in ((256, 1, synth.scene_octree(7, 8)),
                              (336, 2, synth.scene_octree(7, 8, transform=synth.rotation([0, 1, 0], 0.5), scale=0.95))):
        model = synth.siren_tmlp(8, width, seed=seed)
        m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
        m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
        ws = m.workspace(n)
        fws = m.workspace(0)
        y_ref = oracle.query(model, tree, upts)
        yf_ref = oracle.full_depth(model, upts[:20000])
        entry = {}
        for prec in (("fp32", "bf16", "fp8") if width == 336 else ("bf16", "fp8")):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            for _ in range(2):
                m.query(x, precision=prec, out=out, workspace=ws)
            torch.cuda.synchronize()
            counts = np.array(m.stats(ws)["count"][:9], np.int64)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            mlp = []
            t0.record(stream)
            for _ in range(steps):
                m.query(x, precision=prec, out=out, workspace=ws, events=ev)
            t1.record(stream)
            torch.cuda.synchronize()
            sand_ms = t0.elapsed_time(t1) / steps
            mlp_ms = ev[1].elapsed_time(ev[2])
            m.query(x, precision=prec, full_depth=True, out=out, workspace=fws)
            torch.cuda.synchronize()
            t0.record(stream)
            for _ in range(2):
                m.query(x, precision=prec, full_depth=True, out=out, workspace=fws)
            t1.record(stream)
            torch.cuda.synchronize()
            full_ms = t0.elapsed_time(t1) / 2
            flops = float((flops_per_point(np.arange(9), width, False) * counts).sum())
            full_flops = float(flops_per_point(np.array([8]), width, False)[0]) * n
            uy = m.query(ux, precision=prec).double().cpu().numpy()
            e = np.abs(uy - y_ref)
            ufy = m.query(ux[:20000], precision=prec, full_depth=True).double().cpu().numpy()
            # the co-bound of these modes: one hardware sine per unit and row-layer (Eq. 2)
            sines = float((np.arange(9) * width * counts).sum())
            sine_frac = sines / (mlp_ms / 1e3) / sine_rate if sine_rate else None
            entry[prec] = {"sand_queries_per_s": n / (sand_ms / 1e3), "full_depth_queries_per_s": n / (full_ms / 1e3),
                           "sine_pipe_frac_sand": sine_frac,
                           "sand_ms": sand_ms, "full_ms": full_ms,
                           "tmlp_tflops_sand": flops / (mlp_ms / 1e3) / 1e12,
                           "tflops_full_depth": full_flops / (full_ms / 1e3) / 1e12,
                           "max_abs_err": float(e.max()), "rms_err": float(np.sqrt((e ** 2).mean())),
                           "max_abs_err_full_depth_20k": float(np.abs(ufy - yf_ref).max())}
        res["8x%d" % width] = entry
        m.free()
    return res


def trace_bench(sand, model, tree, local: int, steps: int, precision: str = "fp32"):
    """Sphere tracing of a 1920 x 1080 pinhole image (vertical FOV 45 degrees, eye on a radius-2.5
    orbit at azimuth 30, elevation 20, looking at the origin), at most 64 SAND queries per ray,
    hit at |y| < 1e-4, then the input gradient (normal) at the hits."""
    import torch
    eye, dirs = synth.pinhole_rays(1920, 1080, fov_y_deg=45.0, radius=2.5, azimuth_deg=30.0, elevation_deg=20.0)
    e, d = torch.from_numpy(eye).cuda(), torch.from_numpy(dirs).cuda()
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    stream = torch.cuda.current_stream()
    res = {"rays": len(dirs), "max_steps": 64, "hit_eps": 1e-4, "precision": precision,
           "normals": "gradient on the tensor cores (float32 split mode, value and three tangent rows per point)"}
    for normals in (False, True):
        for _ in range(2):
            out = m.sphere_trace(e, d, max_steps=64, hit_eps=1e-4, precision=precision, normals=normals)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            out = m.sphere_trace(e, d, max_steps=64, hit_eps=1e-4, precision=precision, normals=normals)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        res["ms_with_normals" if normals else "ms"] = ms
    _, st, ks, _ = out
    st, ks = st.cpu().numpy(), ks.cpu().numpy()
    q = int(ks.astype(np.int64).sum())
    res.update({"sdf_queries": q, "queries_per_s": q / (res["ms"] / 1e3), "rays_per_s": len(dirs) / (res["ms"] / 1e3),
                "hits": int((st == 1).sum()), "missed": int((st == 0).sum()), "step_limit": int((st == 2).sum()),
                "normal_pass_ms": res["ms_with_normals"] - res["ms"],
                "steps_histogram_16": np.bincount(np.minimum(ks, 64) // 4, minlength=17).tolist()})
    m.free()
    return res


def map_build_bench(sand, model, local: int, steps: int, label: str, rs=(1.5e-4, 1e-2)):
    """The network-depth map from the network (Eq. 5-7) for the level-7 scene octree: Eq. 5 on a
    4^3 lattice per near leaf, max-pooled per leaf, float32 mode, at the paper's r = 1.5e-4 and a
    looser r for a briefly trained network."""
    import torch
    tree = synth.scene_octree(7, N_LAYERS, far_field=True)
    near = ((tree.child < 0) & (tree.depth > 0)).astype(np.uint8)
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    n_near = int(near.sum())
    res = {"model": label, "octree": "scene, level 7, far field", "near_leaves": n_near, "samples_per_leaf": 64,
           "samples": n_near * 64}
    for r in rs:
        got = m.build_depth_map(tree.max_level, tree.child, near, samples_per_axis=4, r=r)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            got = m.build_depth_map(tree.max_level, tree.child, near, samples_per_axis=4, r=r)
        dt = (time.perf_counter() - t0) / steps
        res["r=%g" % r] = {"ms": dt * 1e3, "samples_per_s": n_near * 64 / dt,
                           "depth_histogram": np.bincount(got[near.astype(bool)], minlength=N_LAYERS + 1).tolist()}
    m.free()
    return res


def trained_scene_model(sand, local: int, steps: int):
    """The benchmark's 8 x 256 SIREN after `steps` training steps (sand_train_step, Adam at the
    paper's learning rate 1e-4) on a 100,000-point batch of the analytic scene (60 % surface,
    40 % jittered), so that Eq. 5 and the dynamic exit see tails that approach the SDF."""
    import dataclasses
    import torch
    from paper_2604_25936_gb300.binding import Trainer
    model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED)
    pts, gt = synth.training_batch(100000, seed=22)
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    tr = Trainer(m, max_points=len(pts))
    x, t = torch.from_numpy(pts).cuda(), torch.from_numpy(gt).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    for _ in range(steps):
        tr.step(x, t, loss=loss)
    torch.cuda.synchronize()
    tr.status()
    flat = tr.params()
    final = float(loss.item())
    tr.close()
    m.free()
    parts, o = {}, 0
    L, W = N_LAYERS, WIDTH
    for name, shape in (("W1", (W, 3)), ("b1", (W,)), ("Wh", (L - 1, W, W)), ("bh", (L - 1, W)),
                        ("tail_w", (L, 2, W)), ("tail_b", (L, 2))):
        k = int(np.prod(shape))
        parts[name] = flat[o:o + k].reshape(shape).astype(np.float32)
        o += k
    return dataclasses.replace(model, **parts), final


def dynamic_bench(sand, model, x, n: int, local: int, steps: int):
    """The octree-free dynamic exit of Table 6 on the benchmark lattice (no depth map), at the
    paper's r = 1.5e-4 and at r = 0.05, float32 mode."""
    import torch
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    stream = torch.cuda.current_stream()
    res = {"lattice_points": n, "note": "rows stop at the first tail |t_i| < r; a 128-row tile stops when all its rows have"}
    for r in (1.5e-4, 0.05):
        for _ in range(2):
            y, el = m.query_dynamic(x, r=r)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            y, el = m.query_dynamic(x, r=r)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        res["r=%g" % r] = {"ms": ms, "queries_per_s": n / (ms / 1e3),
                           "exit_layer_histogram": torch.bincount(el.long(), minlength=N_LAYERS + 1).tolist()}
    m.free()
    return res


def grad_bench(sand, m, x, ws, n: int, steps: int):
    """SDF and input gradient (a6) of the SAND query on the benchmark lattice: the tensor-core
    path (value and three tangent rows per point, 32 points per 128-row tile) at float32 and
    bf16, and the CUDA-core kernel beside them."""
    import torch
    stream = torch.cuda.current_stream()
    res = {}
    for prec in ("fp32", "bf16", "fp32_simt"):
        for _ in range(2):
            y, g = m.query_grad(x, precision=prec, workspace=ws)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            y, g = m.query_grad(x, precision=prec, workspace=ws)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        res[prec] = {"ms": round(ms, 4), "queries_per_s": n / (ms / 1e3)}
    res["kernels"] = {"fp32": "tmlp_tc_kernel<split, GRAD>", "bf16": "tmlp_tc_kernel<bf16, GRAD>",
                      "fp32_simt": "tmlp_simt_kernel<GRAD>"}
    return res


def run_profile_case(args):
    """The same model and map as the benchmark on a smaller point set, for ncu captures."""
    import torch
    import paper_2604_25936_gb300 as sand
    from paper_2604_25936_gb300 import build as sand_build
    sand_build.build()
    model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED)
    tree = synth.scene_octree(7, N_LAYERS)
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=0)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    full = args.profile == "full"
    pts = synth.uniform_points(args.grid ** 3, seed=1) if full else synth.lattice(args.grid)
    x = torch.from_numpy(pts).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(args.warmup + args.steps):
        y = m.query(x, precision=args.precision, full_depth=full, events=ev)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "points": len(pts), "precision": args.precision,
                      "tmlp_ms": ev[1].elapsed_time(ev[2]), "max_abs_y": float(y.abs().max())}), flush=True)
    m.free()
    return 0


def _best_ms(fn, reps: int = 10, warm: int = 3) -> float:
    """Shortest of `reps` CUDA-event timings of fn() on the current stream, after `warm` calls."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _sustained_ms(fn, seconds: float = 2.0) -> float:
    """Mean CUDA-event time per call of fn() run back to back for about `seconds`."""
    import torch
    stream = torch.cuda.current_stream()
    calls = max(1, int(seconds * 1e3 / max(_best_ms(fn, reps=2, warm=1), 1e-3)))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(calls):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / calls


def sin_rate(sand, local: int) -> float:
    """Hardware sines per second (sand_probe_rate, one 8 x 256-thread-block wave per SM)."""
    import torch
    nb = torch.cuda.get_device_properties(local).multi_processor_count * 8
    iters = 1 << 14
    sink = torch.empty(nb * sand.binding.PROBE_THREADS, dtype=torch.float32, device="cuda")
    ms = _best_ms(lambda: sand.binding.probe_rate(sand.binding.PROBE_SIN, nb, iters, sink))
    return sand.binding.PROBE_CHAINS * iters * sand.binding.PROBE_THREADS * nb / (ms / 1e3)


def run_peaks(args):
    """Measured throughput of the units behind the kernels' rooflines, on this GPU: cuBLAS
    GEMMs at 8192^3 (bf16, fp16, TF32, float32 SGEMM, FP8 e4m3 through torch._scaled_mm),
    burst (best of 10) and sustained (back to back for 2 s), and the float32 FMA and
    hardware-sine issue rates of sand_probe_rate.  One JSON line."""
    import torch
    import paper_2604_25936_gb300 as sand
    from paper_2604_25936_gb300 import build as sand_build
    sand_build.build()
    torch.cuda.set_device(0)
    props = torch.cuda.get_device_properties(0)
    uuid = None
    try:
        uuid = str(props.uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    res = {"peaks": props.name, "sm_count": props.multi_processor_count, "gemm_n": 8192}
    N = 8192
    flop = 2.0 * N ** 3
    g = torch.Generator(device="cuda").manual_seed(0)
    a32 = torch.randn(N, N, device="cuda", generator=g)
    b32 = torch.randn(N, N, device="cuda", generator=g)
    cases = {"bf16": lambda: torch.matmul(a16b, b16b), "fp16": lambda: torch.matmul(a16h, b16h),
             "tf32": lambda: torch.matmul(a32, b32), "fp32_sgemm": lambda: torch.matmul(a32, b32)}
    a16b, b16b = a32.bfloat16(), b32.bfloat16()
    a16h, b16h = a32.half(), b32.half()
    for name, fn in cases.items():
        torch.backends.cuda.matmul.allow_tf32 = name == "tf32"
        try:
            burst = _best_ms(fn)
            sus = _sustained_ms(fn)
            res[name + "_tflops"] = round(flop / (burst / 1e3) / 1e12, 1)
            res[name + "_tflops_sustained"] = round(flop / (sus / 1e3) / 1e12, 1)
        except Exception as e:  # a library path missing in the installed torch
            res[name + "_tflops"] = None
            res[name + "_error"] = str(e)[:200]
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a8 = a32.clamp(-8, 8).to(torch.float8_e4m3fn)
        b8 = b32.clamp(-8, 8).to(torch.float8_e4m3fn).t().contiguous().t()  # column-major second operand
        one = torch.ones((), device="cuda")
        fn = lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        burst, sus = _best_ms(fn), _sustained_ms(fn)
        res["fp8_tflops"] = round(flop / (burst / 1e3) / 1e12, 1)
        res["fp8_tflops_sustained"] = round(flop / (sus / 1e3) / 1e12, 1)
    except Exception as e:
        res["fp8_tflops"] = None
        res["fp8_error"] = str(e)[:200]
    del a32, b32, a16b, b16b, a16h, b16h
    nb = props.multi_processor_count * 8
    sink = torch.empty(nb * sand.binding.PROBE_THREADS, dtype=torch.float32, device="cuda")
    it = 1 << 16
    ms = _best_ms(lambda: sand.binding.probe_rate(sand.binding.PROBE_FFMA, nb, it, sink))
    res["ffma_tflops"] = round(2.0 * sand.binding.PROBE_CHAINS * it * sand.binding.PROBE_THREADS * nb / (ms / 1e3) / 1e12, 2)
    res["sin_per_s"] = sin_rate(sand, 0)
    ck = clocks.stop()
    res["clocks"] = ck
    if ck and ck.get("sm_mhz"):
        mhz = ck["sm_mhz"]
        res["ffma_per_clk_per_sm"] = round(res["ffma_tflops"] * 1e12 / 2 / (mhz * 1e6) / props.multi_processor_count, 1)
        res["sin_per_clk_per_sm"] = round(res["sin_per_s"] / (mhz * 1e6) / props.multi_processor_count, 2)
    print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sand", choices=["sand", "reference"])
    ap.add_argument("--precision", default="fp32", choices=sorted(TOL))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the 512^3 bf16 / FP8 precision variant and the sphere-tracing workload")
    ap.add_argument("--profile", choices=["sand", "full"], default=None,
                    help="small profiling case: only (warmup + steps) SAND queries on a grid^3 lattice, or full-depth "
                         "queries on grid^3 uniform points; prints one line")
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the bf16 open-loop serving runs at 0.5x and 0.8x of saturation (0 = skip "
                         "serving; the float32 runs take a third of it)")
    ap.add_argument("--sweep-seconds", type=float, default=4.0, help="length of each run of the serving load sweep")
    ap.add_argument("--peaks", action="store_true", help="measure GEMM, FMA and sine peaks of this GPU; prints one line")
    ap.add_argument("--train-only", action="store_true", help="only the training-step measurement; prints one line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.peaks:
        return run_peaks(args)
    if args.profile:
        return run_profile_case(args)
    if args.train_only:
        import torch
        import paper_2604_25936_gb300 as sand
        from paper_2604_25936_gb300 import build as sand_build
        sand_build.build()
        torch.cuda.set_device(0)
        print(json.dumps({"training": train_bench(sand, 0, max(3, args.steps))}), flush=True)
        return 0

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2604_25936_gb300 as sand
    from paper_2604_25936_gb300 import build as sand_build
    sand_build.build()
    prec = args.precision
    W = max(3, args.warmup)
    K = max(1, args.steps)

    model = synth.siren_tmlp(N_LAYERS, WIDTH, seed=SEED)
    tree = synth.scene_octree(7, N_LAYERS)
    pts = synth.lattice(GRID)
    n = len(pts)
    m = sand.Model.from_params(*model.header_ints(), model.omega0, model.flat(), device=local)
    m.set_depth_map(tree.max_level, tree.n_layers, tree.child, tree.depth, tree.far)
    x = torch.from_numpy(pts).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ws = m.workspace(n)
    stream = torch.cuda.current_stream()

    def sand_step(events=None):
        m.query(x, precision=prec, out=out, workspace=ws, events=events)

    for _ in range(W):
        sand_step()
    torch.cuda.synchronize()
    stats = m.stats(ws)
    counts = np.array(stats["count"][:N_LAYERS + 1], np.int64)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(K):
        sand_step(ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end) / K
    mlp_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    pre_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    ms = 1e3 * max_over_ranks(ms / 1e3, world, "cuda")
    value = job_throughput(n, world, ms / 1e3)

    # ---- full-depth baseline: the same T-MLP to layer L at every point
    fout = torch.empty(n, dtype=torch.float32, device="cuda")
    fws = m.workspace(0)
    Kf = max(2, K // 4)
    for _ in range(2):
        m.query(x, precision=prec, full_depth=True, out=fout, workspace=fws)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(Kf):
        m.query(x, precision=prec, full_depth=True, out=fout, workspace=fws)
    f1.record(stream)
    torch.cuda.synchronize()
    full_ms = 1e3 * max_over_ranks(f0.elapsed_time(f1) / Kf / 1e3, world, "cuda")
    full_value = job_throughput(n, world, full_ms / 1e3)

    # ---- error against the oracle on a sample (the "stated error")
    err = err_full = None
    if rank == 0:
        import oracle
        idx = synth.sample_indices(n, 20000, seed=11)
        y_ref = oracle.query(model, tree, pts[idx])
        err = float(np.abs(out.cpu().numpy()[idx].astype(np.float64) - y_ref).max())
        yf_ref = oracle.full_depth(model, pts[idx[:5000]])
        err_full = float(np.abs(fout.cpu().numpy()[idx[:5000]].astype(np.float64) - yf_ref).max())

    # ---- end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    hp = torch.from_numpy(pts).pin_memory()
    ho = torch.empty(n, dtype=torch.float32).pin_memory()
    for _ in range(3):
        m.query_host(hp, out=ho, precision=prec)
    # host wall-clock over about 0.1 s: a shorter window is at the mercy of one hiccup of the
    # host thread that drives the copies
    Ke = max(10, K)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        m.query_host(hp, out=ho, precision=prec)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / Ke, world, "cuda")
    e2e_value = job_throughput(n, world, e2e_s)

    # ---- roofline of the dominant kernel (the T-MLP kernel)
    pk, pk_src = peaks()
    net_flops = float((flops_per_point(np.arange(N_LAYERS + 1), WIDTH, False) * counts).sum())
    mlp_avg = sum(mlp_ms) / len(mlp_ms)
    achieved = net_flops / (mlp_avg / 1e3) / 1e12
    if prec == "fp32_simt":
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        peak = sm_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": kernel_traffic(prec), "kernel": KERNEL_NAME[prec],
                "peak_source": "derived: %d SMs x 128 FP32 FMA/clk x 2 FLOP x %.0f MHz (max SM clock, %s)"
                               % (sm_count, pk.get("sm_max_mhz", 2070.0), pk_src)}
    else:
        base = pk.get("bf16_tflops_sustained", 1700.0)
        ratio = {"fp32": 1.0 / 3.0, "fp16": 1.0, "bf16": 1.0, "fp8": 2.0}[prec]
        peak = base * ratio
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": kernel_traffic(prec), "kernel": KERNEL_NAME[prec],
                "peak_source": "%s bf16 sustained %.1f TFLOP/s x %.3g (%s)" % (pk_src, base, ratio, prec)}
    # the epilogue's co-bound: one hardware sine per unit per row-layer (Eq. 2), against the
    # issue rate sand_probe_rate measures on this GPU in this run
    sines = float((np.arange(N_LAYERS + 1) * WIDTH * counts).sum())
    sr = sin_rate(sand, local)
    epi = {"unit": "sines/s", "achieved": sines / (mlp_avg / 1e3), "peak": sr, "frac": sines / (mlp_avg / 1e3) / sr,
           "sines_per_launch": sines, "peak_source": "sand_probe_rate(SAND_PROBE_SIN), measured in this run"}

    # ---- serving: continuous batching over three resident models (rank 0 only)
    serve = None
    if rank == 0 and args.serve_seconds > 0:
        smodels = serve_models(sand)
        pool = serve_requests(40, seed=5)
        serve = {"bf16": serve_bench(sand, smodels, "bf16", pool, args.serve_seconds, args.sweep_seconds),
                 "fp32": serve_bench(sand, smodels, "fp32", pool, args.serve_seconds / 3, args.sweep_seconds)}
        for sm in smodels:
            sm.free()

    tr = None
    if rank == 0 and not args.no_variants:
        tr = trace_bench(sand, model, synth.scene_octree(7, N_LAYERS, far_field=True), local, max(3, K // 4))

    gradb = None
    if rank == 0 and not args.no_variants:
        gradb = grad_bench(sand, m, x, ws, n, max(2, K // 8))

    dynb = None
    if rank == 0 and not args.no_variants:
        dynb = dynamic_bench(sand, model, x, n, local, max(2, K // 8))

    mapb = None
    if rank == 0 and not args.no_variants:
        trained, trained_loss = trained_scene_model(sand, local, 1000)
        mapb = {"random_init": map_build_bench(sand, model, local, max(2, K // 8), "random SIREN init"),
                "trained": map_build_bench(sand, trained, local, max(2, K // 8),
                                           "1000 training steps (loss %.4g)" % trained_loss)}
        dynb = {"random_init": dynb, "trained": dynamic_bench(sand, trained, x, n, local, max(2, K // 8))}

    variant = None
    if rank == 0 and not args.no_variants:
        variant = precision_variant(sand, local, max(3, K // 4), sine_rate=sr)

    deepb = None
    if rank == 0 and not args.no_variants:
        deepb = deep_map_bench(sand, local, max(3, K // 4))

    trainb = None
    if rank == 0 and not args.no_variants:
        trainb = train_bench(sand, local, max(3, K // 2))

    paperv = None
    if rank == 0 and not args.no_variants and prec != "fp32_simt":
        paperv = paper_variants(sand, local, max(3, K // 4), prec, roof["peak"], pk.get("hbm_gbs", 6800.0))

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(model, tree, pts)

    hist = {str(d): int(c) for d, c in enumerate(counts)}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "queries/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE[prec],
        "data": "synthetic: random SIREN-init 8x256 T-MLP (seed 1), analytic-scene level-7 octree, marching-cubes lattice",
        "config": {"workload": WORKLOAD,
                   "global_batch": world * n, "points_per_gpu": n, "precision": prec,
                   "l2": "inputs larger than L2 (201 MB of points per step), no flush",
                   "parallelism": "replicas (one full lattice per GPU)"},
        "full_depth": {"value": full_value, "unit": "queries/s", "ms_per_step": full_ms,
                       "speedup_sand_vs_full": value / full_value, "max_abs_err_vs_oracle_5k": err_full},
        "max_abs_err_vs_oracle_20k": err,
        "tolerance": TOL[prec],
        "stage_ms": {"lookup_bin": sum(pre_ms) / K, "tmlp": mlp_avg},
        "hbm_stages": hbm_stages(n, int(counts[0]), sum(pre_ms) / K, pk.get("hbm_gbs", 6800.0)),
        "exit_layer_histogram": hist,
        "roofline": roof,
        "epilogue_pipe": epi,
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 4 * n},
        "gpu_launches": 4 * K,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "serve": serve,
        "precision_variant": variant,
        "paper_variants": paperv,
        "training": trainb,
        "deep_map": deepb,
        "sphere_trace": tr,
        "depth_map_build": mapb,
        "dynamic_exit": dynb,
        "gradient": gradb,
        "serve_p99_ms": (serve or {}).get("bf16", {}).get("load_0.8", {}).get("p99_ms"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.free()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
