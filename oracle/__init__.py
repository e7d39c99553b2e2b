"""FP64 CPU oracle for the SAND query path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the library: they share no code, only the generated
inputs of ``synth``.

The arithmetic lives in ``sand_oracle.c`` (plain per-point double-precision
loops, OpenMP over points); this module compiles it with gcc on first use
(``-O2 -ffp-contract=off``, no fast-math) and marshals numpy arrays.
Functions follow SAND (arxiv 2604.25936): ``lookup`` the octree of Sec. 3.2 /
Eq. 7 with the level-of-detail clamp of Sec. 3.4, ``evaluate`` the T-MLP of
Eq. 2 / Eq. 3 to given exit layers, ``query`` the whole inference procedure
of Sec. 3.4, each optionally with the input gradient by reverse-mode chain
rule.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sand_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's shared library (gcc, OpenMP) if missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_lookup.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int64, ctypes.c_int, P, P]
            lib.oracle_eval.argtypes = [P, ctypes.c_double, P, P, ctypes.c_int64, P, ctypes.c_int, P, P, P]
            lib.oracle_query.argtypes = [P, ctypes.c_double, P, ctypes.c_int, P, P, P, P, ctypes.c_int64,
                                         ctypes.c_int, P, P, P]
            lib.oracle_preact_margin.argtypes = [P, ctypes.c_double, P, P, ctypes.c_int64, P, ctypes.c_int, P]
            lib.oracle_train_grad.argtypes = [P, ctypes.c_double, P, P, P, ctypes.c_int64, P, P]
            lib.oracle_param_count.argtypes = [P]
            lib.oracle_param_count.restype = ctypes.c_longlong
            lib.oracle_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """OpenMP threads the oracle runs on."""
    return int(_load().oracle_threads())


def _model_args(model):
    hdr = np.ascontiguousarray(np.array(model.header_ints(), np.int32))
    params = np.ascontiguousarray(model.flat(), np.float32)
    n_expect = _load().oracle_param_count(_ptr(hdr))
    if params.size != n_expect:
        raise ValueError("parameter block has %d floats, header implies %d" % (params.size, n_expect))
    return hdr, float(model.omega0), params


def _pts(points):
    p = np.ascontiguousarray(np.asarray(points, np.float32).reshape(-1, 3))
    return p


def lookup(octree, points, max_depth: int = 0):
    """Exit layer (int32, -1 for NaN points) and stored far value (float64) per point."""
    p = _pts(points)
    n = p.shape[0]
    d = np.empty(n, np.int32)
    f = np.empty(n, np.float64)
    child = np.ascontiguousarray(octree.child, np.int32)
    dep = np.ascontiguousarray(octree.depth, np.uint8)
    far = np.ascontiguousarray(octree.far, np.float32)
    rc = _load().oracle_lookup(int(child.size), _ptr(child), _ptr(dep), _ptr(far), _ptr(p), n,
                               int(max_depth), _ptr(d), _ptr(f))
    if rc:
        raise RuntimeError("oracle_lookup failed: %d" % rc)
    return d, f


def evaluate(model, points, depth, grad: bool = False, all_tails: bool = False):
    """T-MLP outputs y_d at exit layer(s) `depth` (int or int array; <= 0 gives 0).

    Returns y (float64 [n]); plus grad [n,3] if grad; plus ys [n,L] (y_1..y_d,
    zero beyond d) if all_tails.
    """
    hdr, w0, params = _model_args(model)
    p = _pts(points)
    n = p.shape[0]
    y = np.empty(n, np.float64)
    g = np.empty((n, 3), np.float64) if grad else None
    ys = np.empty((n, model.n_layers), np.float64) if all_tails else None
    if np.isscalar(depth) or np.ndim(depth) == 0:
        darr, cd = None, int(depth)
    else:
        darr, cd = np.ascontiguousarray(np.asarray(depth, np.int32)), 0
    rc = _load().oracle_eval(_ptr(hdr), w0, _ptr(params), _ptr(p), n, _ptr(darr), cd, _ptr(y), _ptr(g), _ptr(ys))
    if rc:
        raise RuntimeError("oracle_eval failed: %d" % rc)
    out = [y]
    if grad:
        out.append(g)
    if all_tails:
        out.append(ys)
    return out[0] if len(out) == 1 else tuple(out)


def preact_margin(model, points, depth):
    """Per point, the smallest |u_l[j]| over the pre-activations u_l = W_l h_{l-1} + b_l of
    layers 1..d (Eq. 1; +inf where d <= 0).  Where a ReLU network's gradient is compared
    across two evaluations, points whose margin exceeds the pre-activation error take the
    same ReLU decisions in both."""
    hdr, w0, params = _model_args(model)
    p = _pts(points)
    n = p.shape[0]
    out = np.empty(n, np.float64)
    if np.isscalar(depth) or np.ndim(depth) == 0:
        darr, cd = None, int(depth)
    else:
        darr, cd = np.ascontiguousarray(np.asarray(depth, np.int32)), 0
    rc = _load().oracle_preact_margin(_ptr(hdr), w0, _ptr(params), _ptr(p), n, _ptr(darr), cd, _ptr(out))
    if rc:
        raise RuntimeError("oracle_preact_margin failed: %d" % rc)
    return out


def query(model, octree, points, max_depth: int = 0, grad: bool = False, exit_layers: bool = False):
    """SAND inference (Sec. 3.4): y per point (float64); optionally grad [n,3]
    and exit layers (int32, -1 for NaN points)."""
    hdr, w0, params = _model_args(model)
    p = _pts(points)
    n = p.shape[0]
    y = np.empty(n, np.float64)
    g = np.empty((n, 3), np.float64) if grad else None
    d = np.empty(n, np.int32) if exit_layers else None
    child = np.ascontiguousarray(octree.child, np.int32)
    dep = np.ascontiguousarray(octree.depth, np.uint8)
    far = np.ascontiguousarray(octree.far, np.float32)
    rc = _load().oracle_query(_ptr(hdr), w0, _ptr(params), int(child.size), _ptr(child), _ptr(dep), _ptr(far),
                              _ptr(p), n, int(max_depth), _ptr(y), _ptr(g), _ptr(d))
    if rc:
        raise RuntimeError("oracle_query failed: %d" % rc)
    out = [y]
    if grad:
        out.append(g)
    if exit_layers:
        out.append(d)
    return out[0] if len(out) == 1 else tuple(out)


def full_depth(model, points, grad: bool = False):
    """The plain T-MLP evaluated to its last layer at every point (no depth map)."""
    return evaluate(model, points, model.n_layers, grad=grad)


# ---------------------------------------------------------------------------------------------
# Network-depth map from the network (Sec. 3.2, Eq. 5-7)
# ---------------------------------------------------------------------------------------------
def leaf_cells(child):
    """Every leaf of a pointer octree over [-1, 1]^3 (root = node 0, the children of a node
    consecutive in octant order ix | iy << 1 | iz << 2) as rows (node, level, ix, iy, iz):
    the leaf's cell is [-1 + 2 ix / 2^level, -1 + 2 (ix + 1) / 2^level) per axis."""
    child = np.asarray(child)
    out = []
    stack = [(0, 0, 0, 0, 0)]
    while stack:
        n, lv, ix, iy, iz = stack.pop()
        c = int(child[n])
        if c < 0:
            out.append((n, lv, ix, iy, iz))
            continue
        for o in range(8):
            stack.append((c + o, lv + 1, 2 * ix + (o & 1), 2 * iy + ((o >> 1) & 1), 2 * iz + ((o >> 2) & 1)))
    return np.array(sorted(out), np.int64).reshape(-1, 5)


def leaf_samples(cells, k: int):
    """The k^3 cell-centred lattice of sample points in each leaf cell, float32 [n_leaves * k^3, 3]
    (leaf-major, x fastest within a leaf): x = lo + (s + 1/2) side / k.  For a power-of-two k
    every value is exact in float32."""
    lv = cells[:, 1].astype(np.float64)
    side = 2.0 / np.exp2(lv)
    lo = -1.0 + cells[:, 2:5].astype(np.float64) * side[:, None]
    s = np.arange(k, dtype=np.float64)
    sz, sy, sx = np.meshgrid(s, s, s, indexing="ij")
    sub = np.stack([sx.ravel(), sy.ravel(), sz.ravel()], axis=1)  # [k^3, 3], x fastest
    pts = lo[:, None, :] + (sub[None, :, :] + 0.5) * (side / k)[:, None, None]
    return pts.reshape(-1, 3).astype(np.float32)


def required_depth(ys, r: float, near: bool = True):
    """Eq. 5 per point from its cumulative outputs ys [n, L] (y_1 .. y_L): the smallest i with
    sign(y_i) = sign(y_L) (sign(0) taken as +1), and, near the surface, |y_L - y_i| < r.
    i = L always qualifies, so every point gets a depth in 1 .. L."""
    ys = np.asarray(ys, np.float64)
    yl = ys[:, -1:]
    ok = np.where(ys >= 0, 1, -1) == np.where(yl >= 0, 1, -1)
    if near:
        ok &= np.abs(yl - ys) < r
    return np.argmax(ok, axis=1).astype(np.int64) + 1


def depth_map_from_network(model, child, near, k: int = 4, r: float = 1.5e-4, far_sign: bool = False):
    """Eq. 6: the depth of a near leaf (near[node] != 0) is the maximum of Eq. 5 over its k^3
    sample points; far leaves keep depth 0 (Eq. 7: they answer with their stored value), or,
    with far_sign, get the maximum over their samples of the sign-only case of Eq. 5.
    Returns (depth per node as uint8, sample points, their Eq. 5 depths, leaf row per sample,
    the samples' y_1 .. y_L in float64)."""
    near = np.asarray(near)
    cells = leaf_cells(child)
    use = np.array([bool(near[c[0]]) or far_sign for c in cells], bool)
    cells = cells[use]
    pts = leaf_samples(cells, k)
    _, ys = evaluate(model, pts, model.n_layers, all_tails=True)
    kk = k ** 3
    leaf_row = np.repeat(np.arange(len(cells)), kk)
    is_near = np.repeat(np.array([bool(near[c[0]]) for c in cells], bool), kk)
    d = np.where(is_near, required_depth(ys, r, True), required_depth(ys, r, False))
    depth = np.zeros(len(child), np.uint8)
    for row, c in enumerate(cells):
        depth[c[0]] = int(d[row * kk:(row + 1) * kk].max())
    return depth, pts, d, leaf_row, ys


def dynamic_exit(model, points, r: float):
    """The octree-free dynamic inference of Table 6: a point runs layer by layer and stops at
    the first layer i whose tail |t_i| = |y_i - y_{i-1}| < r (y_0 = 0), or at layer L.
    Returns (y at that layer, the layer as int64, all y_1 .. y_L in float64)."""
    _, ys = evaluate(model, points, model.n_layers, all_tails=True)
    t = np.diff(np.concatenate([np.zeros((ys.shape[0], 1)), ys], axis=1), axis=1)
    stop = np.abs(t) < r
    stop[:, -1] = True
    d = np.argmax(stop, axis=1) + 1
    return ys[np.arange(len(d)), d - 1], d.astype(np.int64), ys


# ---------------------------------------------------------------------------------------------
# Training (Sec. 3.3): the loss over every tail (Eq. 4 with the L1 SDF loss of Eq. 8) and Adam
# ---------------------------------------------------------------------------------------------
def train_grad(model, points, gt):
    """The training loss L = sum_i (1/n) sum_x |y_i(x) - gt(x)| (Eq. 4 / Eq. 8) and its gradient
    with respect to every parameter, as a float64 vector in the parameter-block order of
    model.flat() (a Fourier matrix is not trained: its entries are 0).  |r|' = sign(r), sign(0)
    = 0.  Returns (loss, grad)."""
    hdr, w0, params = _model_args(model)
    p = _pts(points)
    n = p.shape[0]
    t = np.ascontiguousarray(np.asarray(gt, np.float32).reshape(-1))
    if t.size != n or n == 0:
        raise ValueError("need one target per point and at least one point")
    loss = np.zeros(1, np.float64)
    grad = np.empty(params.size, np.float64)
    rc = _load().oracle_train_grad(_ptr(hdr), w0, _ptr(params), _ptr(p), _ptr(t), n, _ptr(loss), _ptr(grad))
    if rc:
        raise RuntimeError("oracle_train_grad failed: %d" % rc)
    return float(loss[0]), grad


def adam_step(params, grad, m, v, step: int, lr: float = 1e-4, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) in float64, the optimiser of Sec. 4.1:
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;  p <- p - lr (m / (1 - b1^t)) /
    (sqrt(v / (1 - b2^t)) + eps), t = step >= 1.  Returns the new (params, m, v)."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v
