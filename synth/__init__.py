"""Seeded synthetic inputs for the SAND query path.

This module only *generates inputs*: T-MLP weights drawn from seeded
generators, octree depth maps built from analytic signed-distance scenes,
query lattices, uniform samples, camera rays and the on-disk formats that
carry them.  It contains none of the arithmetic of the query path itself
(no octree lookup, no T-MLP evaluation, no gradient): both the FP64 oracle
(``oracle/``) and the CUDA library (``paper_2604_25936_gb300``) consume the
same generated arrays or files, and each parses and evaluates them with its
own code.

Paper context (SAND, arxiv 2604.25936):
  * T-MLP parameters follow Eq. 2 (a tail per hidden layer) and, for the
    multiplicative variant, Eq. 3 (tails i >= 2 are products of two affine
    maps); the first tail is always affine.
  * The depth map is the octree of Sec. 3.2: a node is split while its cell
    intersects the shape and its level is below the maximum; a cell
    "intersects" when the distance from its centre to the surface is at
    most half its diagonal (Sec. 4.1).  Leaves carry either an exit layer
    or, for far leaves in the far-field variant, the SDF value at the leaf
    centre (Eq. 7).
  * Query grids are marching-cubes lattices (512^3 in Sec. 4.1).
Since the paper's trained weights and meshes are not available, weights
are random SIREN-initialised and exit layers come from a fixed rule on an
analytic SDF (distance bands plus a curvature proxy) instead of Eq. 5.
"""
from __future__ import annotations

import dataclasses
import math
import struct
from typing import Callable, Optional

import numpy as np

TAIL_LINEAR, TAIL_MULT = 0, 1
ACT_SINE, ACT_RELU, ACT_FINER = 0, 1, 2
ENC_NONE, ENC_FOURIER = 0, 1

MODEL_MAGIC = b"TMLP"
MAP_MAGIC = b"SDMO"
FORMAT_VERSION = 1


# --------------------------------------------------------------------------
# T-MLP parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass
class TMLP:
    """FP32 master parameters of a T-MLP (Eq. 2 / Eq. 3).

    Shapes (L = n_layers hidden layers, W = width, D = in_dim):
      enc_B  [m, 3]      Fourier-feature matrix (encoder == ENC_FOURIER) or None
      W1     [W, D]      first hidden layer, rows = output neurons
      b1     [W]
      Wh     [L-1, W, W] hidden layers 2..L, Wh[l-2] is [out, in]
      bh     [L-1, W]
      tail_w [L, 2, W]   tail i uses row 0 (linear) or rows 0 and 1 (mult, i >= 2)
      tail_b [L, 2]
    """
    n_layers: int
    width: int
    in_dim: int
    tail_kind: int
    activation: int
    encoder: int
    n_freq: int
    omega0: float
    enc_B: Optional[np.ndarray]
    W1: np.ndarray
    b1: np.ndarray
    Wh: np.ndarray
    bh: np.ndarray
    tail_w: np.ndarray
    tail_b: np.ndarray

    def flat(self) -> np.ndarray:
        """Parameters concatenated in the canonical order of the C-ABI:
        enc_B, W1, b1, Wh, bh, tail_w, tail_b (row-major float32)."""
        parts = []
        if self.encoder == ENC_FOURIER:
            parts.append(self.enc_B.reshape(-1))
        parts += [self.W1.reshape(-1), self.b1.reshape(-1), self.Wh.reshape(-1),
                  self.bh.reshape(-1), self.tail_w.reshape(-1), self.tail_b.reshape(-1)]
        return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))

    def header_ints(self):
        return (self.n_layers, self.width, self.in_dim, self.tail_kind,
                self.activation, self.encoder, self.n_freq)


def _f32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64).astype(np.float32)


def siren_tmlp(n_layers: int, width: int, seed: int, tail_kind: int = TAIL_LINEAR,
               omega0: float = 30.0) -> TMLP:
    """Random SIREN-initialised T-MLP.

    First layer W ~ U(-1/3, 1/3) (fan-in 3); hidden W ~ U(+-sqrt(6/W)/omega0);
    biases ~ U(+-1/sqrt(fan_in)); tail weights ~ U(+-sqrt(6/W)/omega0), tail
    biases 0.  Drawn from one PCG64(seed) stream in float64 in the order
    W1, b1, (W_l, b_l for l = 2..L), (tail rows 0,1 for l = 1..L), then
    rounded to float32.  Tail 1 is always affine: its second row is zero.
    """
    L, W = n_layers, width
    g = np.random.Generator(np.random.PCG64(seed))
    W1 = g.uniform(-1.0 / 3.0, 1.0 / 3.0, (W, 3))
    b1 = g.uniform(-1.0 / math.sqrt(3.0), 1.0 / math.sqrt(3.0), W)
    a = math.sqrt(6.0 / W) / omega0
    Wh = np.zeros((L - 1, W, W))
    bh = np.zeros((L - 1, W))
    for l in range(L - 1):
        Wh[l] = g.uniform(-a, a, (W, W))
        bh[l] = g.uniform(-1.0 / math.sqrt(W), 1.0 / math.sqrt(W), W)
    tw = g.uniform(-a, a, (L, 2, W))
    tb = np.zeros((L, 2))
    if tail_kind == TAIL_LINEAR:
        tw[:, 1, :] = 0.0
    else:
        tw[0, 1, :] = 0.0
    return TMLP(L, W, 3, tail_kind, ACT_SINE, ENC_NONE, 0, float(omega0), None,
                _f32(W1), _f32(b1), _f32(Wh), _f32(bh), _f32(tw), _f32(tb))


def finer_tmlp(n_layers: int, width: int, seed: int, tail_kind: int = TAIL_LINEAR, omega0: float = 30.0,
               bias_k: float = 1.0) -> TMLP:
    """Random FINER T-MLP: the SIREN-initialised weights of siren_tmlp(n_layers, width, seed,
    tail_kind, omega0) with the variable-periodic activation sin(omega0 (|z| + 1) z) and the
    first layer's biases redrawn from U(-bias_k, bias_k) (FINER widens that range to reach
    the higher-frequency parts of the activation) from PCG64(seed + 7919) in float64."""
    t = siren_tmlp(n_layers, width, seed, tail_kind=tail_kind, omega0=omega0)
    g = np.random.Generator(np.random.PCG64(seed + 7919))
    return dataclasses.replace(t, activation=ACT_FINER, b1=_f32(g.uniform(-bias_k, bias_k, width)))


def relu_ff_tmlp(n_layers: int, width: int, n_freq: int, sigma: float, seed: int,
                 tail_kind: int = TAIL_LINEAR) -> TMLP:
    """Random ReLU T-MLP on Fourier features gamma(x) = [sin(2 pi B x), cos(2 pi B x)].

    B ~ N(0, sigma^2) of shape [n_freq, 3]; layer weights He-uniform
    U(+-sqrt(6/fan_in)); biases U(+-1/sqrt(fan_in)); tail weights
    U(+-sqrt(6/W)) * 0.1, tail biases 0.  One PCG64(seed) stream, order
    B, W1, b1, hidden layers, tails.
    """
    L, W = n_layers, width
    D = 2 * n_freq
    g = np.random.Generator(np.random.PCG64(seed))
    B = g.normal(0.0, sigma, (n_freq, 3))
    W1 = g.uniform(-math.sqrt(6.0 / D), math.sqrt(6.0 / D), (W, D))
    b1 = g.uniform(-1.0 / math.sqrt(D), 1.0 / math.sqrt(D), W)
    Wh = np.zeros((L - 1, W, W))
    bh = np.zeros((L - 1, W))
    for l in range(L - 1):
        Wh[l] = g.uniform(-math.sqrt(6.0 / W), math.sqrt(6.0 / W), (W, W))
        bh[l] = g.uniform(-1.0 / math.sqrt(W), 1.0 / math.sqrt(W), W)
    tw = g.uniform(-math.sqrt(6.0 / W), math.sqrt(6.0 / W), (L, 2, W)) * 0.1
    tb = np.zeros((L, 2))
    if tail_kind == TAIL_LINEAR:
        tw[:, 1, :] = 0.0
    else:
        tw[0, 1, :] = 0.0
    return TMLP(L, W, D, tail_kind, ACT_RELU, ENC_FOURIER, n_freq, 1.0, _f32(B),
                _f32(W1), _f32(b1), _f32(Wh), _f32(bh), _f32(tw), _f32(tb))


def relu_sphere_tmlp(radius: float, width: int = 8, n_layers: int = 4) -> TMLP:
    """Hand-built ReLU T-MLP with multiplicative tails whose outputs are exact.

    Layer 1 emits [x+, x-, y+, y-, z+, z-, 0...] (ReLU of +-x), layers 2..L
    are identities on those non-negative features.  Tail 1 = -r^2 (bias
    only); tail 2 = (x+ - x-)^2 = x^2, tail 3 = y^2, tail 4 = z^2.  So the
    cumulative outputs are y1 = -r^2, y2 = x^2 - r^2, y3 = x^2 + y^2 - r^2,
    y4 = |x|^2 - r^2 (the implicit sphere) for n_layers = 4.
    """
    assert width >= 6 and n_layers >= 4
    L, W = n_layers, width
    W1 = np.zeros((W, 3))
    for a in range(3):
        W1[2 * a, a] = 1.0
        W1[2 * a + 1, a] = -1.0
    Wh = np.zeros((L - 1, W, W))
    for l in range(L - 1):
        Wh[l] = np.eye(W)
    tw = np.zeros((L, 2, W))
    tb = np.zeros((L, 2))
    tb[0, 0] = -radius * radius
    for l, a in zip((1, 2, 3), (0, 1, 2)):
        tw[l, 0, 2 * a], tw[l, 0, 2 * a + 1] = 1.0, -1.0
        tw[l, 1, 2 * a], tw[l, 1, 2 * a + 1] = 1.0, -1.0
    return TMLP(L, W, 3, TAIL_MULT, ACT_RELU, ENC_NONE, 0, 1.0, None,
                _f32(W1), np.zeros(W, np.float32), _f32(Wh), np.zeros((L - 1, W), np.float32),
                _f32(tw), _f32(tb))


def relu_plane_tmlp(normal, offset: float, width: int = 8, n_layers: int = 2) -> TMLP:
    """Hand-built ReLU T-MLP with affine tails: y1 = n . x - offset exactly
    (tail 1 reads n_a (x_a+ - x_a-)), every later tail is zero."""
    L, W = n_layers, width
    W1 = np.zeros((W, 3))
    for a in range(3):
        W1[2 * a, a] = 1.0
        W1[2 * a + 1, a] = -1.0
    Wh = np.zeros((L - 1, W, W))
    for l in range(L - 1):
        Wh[l] = np.eye(W)
    tw = np.zeros((L, 2, W))
    tb = np.zeros((L, 2))
    for a in range(3):
        tw[0, 0, 2 * a], tw[0, 0, 2 * a + 1] = normal[a], -normal[a]
    tb[0, 0] = -offset
    return TMLP(L, W, 3, TAIL_LINEAR, ACT_RELU, ENC_NONE, 0, 1.0, None,
                _f32(W1), np.zeros(W, np.float32), _f32(Wh), np.zeros((L - 1, W), np.float32),
                _f32(tw), _f32(tb))


def save_tmlp(path: str, m: TMLP) -> None:
    """Model file: 'TMLP', u32 version, 7 x i32 (n_layers, width, in_dim,
    tail_kind, activation, encoder, n_freq), f32 omega0, u64 n_params, then
    n_params little-endian float32 in the canonical order of TMLP.flat()."""
    p = m.flat()
    with open(path, "wb") as f:
        f.write(MODEL_MAGIC)
        f.write(struct.pack("<I7ifQ", FORMAT_VERSION, *m.header_ints(), float(m.omega0), p.size))
        f.write(p.astype("<f4").tobytes())


# --------------------------------------------------------------------------
# Octree depth maps
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Octree:
    """Pointer octree over [-1, 1]^3 stored as node arrays (root = node 0).

    child[i] = -1 for a leaf, else the index of the first of 8 consecutive
    children ordered by octant = ix | iy << 1 | iz << 2 (upper half = 1).
    depth[i] = exit layer of leaf i (0 = far leaf answered by far[i]).
    far[i]   = stored SDF value at the leaf centre (used when depth == 0).
    level[i], centre[i] are kept for inspection and tests only.
    """
    max_level: int
    n_layers: int
    child: np.ndarray
    depth: np.ndarray
    far: np.ndarray
    level: np.ndarray
    centre: np.ndarray

    @property
    def n_nodes(self) -> int:
        return int(self.child.size)


_OCT = np.array([[(o >> 0) & 1, (o >> 1) & 1, (o >> 2) & 1] for o in range(8)], dtype=np.float64)


def build_octree(max_level: int, n_layers: int,
                 split: Callable[[np.ndarray, float, int], np.ndarray],
                 payload: Callable[[np.ndarray, float, int], tuple]) -> Octree:
    """Breadth-first octree build.

    split(centres [k,3], side, level) -> bool[k]   (only asked for level < max_level)
    payload(centres [k,3], side, level) -> (depth uint8[k], far float32[k]) for leaves.
    Nodes are numbered level by level; the 8 children of a node are consecutive.
    """
    child = [np.full(1, -1, np.int64)]
    depth = [np.zeros(1, np.uint8)]
    far = [np.zeros(1, np.float32)]
    level = [np.zeros(1, np.int32)]
    centre = [np.zeros((1, 3))]
    n_total = 1
    lev = 0
    while True:
        cur_c, cur_child, cur_d, cur_f = centre[-1], child[-1], depth[-1], far[-1]
        side = 2.0 / (1 << lev)
        s = np.asarray(split(cur_c, side, lev), bool) if lev < max_level else np.zeros(len(cur_c), bool)
        if (~s).any():
            d, fv = payload(cur_c[~s], side, lev)
            cur_d[~s] = np.asarray(d, np.uint8)
            cur_f[~s] = np.asarray(fv, np.float32)
        k = int(s.sum())
        if k == 0:
            break
        cur_child[s] = n_total + 8 * np.arange(k)
        kids = (cur_c[s][:, None, :] + (2.0 * _OCT[None, :, :] - 1.0) * (side / 4.0)).reshape(-1, 3)
        child.append(np.full(8 * k, -1, np.int64))
        depth.append(np.zeros(8 * k, np.uint8))
        far.append(np.zeros(8 * k, np.float32))
        level.append(np.full(8 * k, lev + 1, np.int32))
        centre.append(kids)
        n_total += 8 * k
        lev += 1
    return Octree(max_level, n_layers, np.concatenate(child).astype(np.int32), np.concatenate(depth),
                  np.concatenate(far), np.concatenate(level), np.concatenate(centre))


def save_octree(path: str, t: Octree) -> None:
    """Depth-map file: 'SDMO', u32 version, i32 max_level, i32 n_layers,
    i32 n_nodes, 6 x f32 bbox (-1,-1,-1, 1,1,1), then child int32[n],
    depth uint8[n] zero-padded to a multiple of 4 bytes, far float32[n]."""
    n = t.n_nodes
    with open(path, "wb") as f:
        f.write(MAP_MAGIC)
        f.write(struct.pack("<I3i6f", FORMAT_VERSION, t.max_level, t.n_layers, n,
                            -1, -1, -1, 1, 1, 1))
        f.write(t.child.astype("<i4").tobytes())
        d = t.depth.astype(np.uint8).tobytes()
        f.write(d + b"\0" * ((-len(d)) % 4))
        f.write(t.far.astype("<f4").tobytes())


# ---- analytic scenes (inputs only: used to build maps, never by the query path)
def sphere_sdf(p: np.ndarray, c, r: float) -> np.ndarray:
    return np.linalg.norm(p - np.asarray(c, np.float64), axis=-1) - r


def torus_y_sdf(p: np.ndarray, c, R: float, r: float) -> np.ndarray:
    q = p - np.asarray(c, np.float64)
    a = np.hypot(q[..., 0], q[..., 2]) - R
    return np.hypot(a, q[..., 1]) - r


def scene_sdf(p: np.ndarray, transform: Optional[np.ndarray] = None, scale: float = 1.0) -> np.ndarray:
    """Union (min) of three spheres and a y-axis torus; optionally evaluated in
    a rotated / scaled frame (p_local = R^T p / scale, d = scale * d_local)."""
    p = np.asarray(p, np.float64)
    if transform is not None:
        p = p @ transform  # row vectors: p R  ==  (R^T p)^T
    p = p / scale
    d = np.minimum.reduce([
        sphere_sdf(p, (-0.35, 0.0, 0.0), 0.30),
        sphere_sdf(p, (0.35, 0.10, 0.0), 0.25),
        sphere_sdf(p, (0.0, -0.30, 0.30), 0.20),
        torus_y_sdf(p, (0.0, 0.35, -0.20), 0.35, 0.08),
    ])
    return d * scale


def hessian_frobenius(f: Callable[[np.ndarray], np.ndarray], c: np.ndarray, h: float) -> np.ndarray:
    """Central finite-difference Hessian Frobenius norm of f at centres c [k,3]."""
    c = np.asarray(c, np.float64)
    f0 = f(c)
    H = np.zeros((len(c), 3, 3))
    E = np.eye(3) * h
    for i in range(3):
        H[:, i, i] = (f(c + E[i]) - 2.0 * f0 + f(c - E[i])) / (h * h)
        for j in range(i + 1, 3):
            v = (f(c + E[i] + E[j]) - f(c + E[i] - E[j]) - f(c - E[i] + E[j]) + f(c - E[i] - E[j])) / (4 * h * h)
            H[:, i, j] = H[:, j, i] = v
    return np.sqrt((H * H).sum(axis=(1, 2)))


def voxel_sphere_octree(level: int = 3, radius: float = 0.5) -> Octree:
    """Dense voxel depth map (complete octree to `level`) with exit layers from
    | |c| - radius | at the voxel centre: < 0.05 -> 4, < 0.15 -> 3, < 0.4 -> 2, else 1."""
    def split(c, side, lev):
        return np.ones(len(c), bool)

    def payload(c, side, lev):
        s = np.abs(np.linalg.norm(c, axis=1) - radius)
        d = np.where(s < 0.05, 4, np.where(s < 0.15, 3, np.where(s < 0.4, 2, 1)))
        return d.astype(np.uint8), np.zeros(len(c), np.float32)
    return build_octree(level, 4, split, payload)


def scene_octree(max_level: int = 7, n_layers: int = 8, far_field: bool = False,
                 transform: Optional[np.ndarray] = None, scale: float = 1.0,
                 hess_threshold: float = 8.0) -> Octree:
    """Adaptive octree of the analytic scene.

    Split rule: |sdf(c)| <= (sqrt(3)/2) * side and level < max_level.
    Leaf exit layer from |sdf(c)|: >= 0.4 -> 1, >= 0.2 -> 2, >= 0.1 -> 3,
    >= 0.05 -> 4, >= 0.025 -> 5, >= h -> 6, else 7 (h = 2 / 2^max_level),
    plus one (capped at n_layers) where the finite-difference Hessian
    Frobenius norm (step h) exceeds hess_threshold.  The layer bands are
    then rescaled to n_layers when n_layers != 8.  With far_field, leaves
    whose cell does not intersect the surface get exit layer 0 and store
    sdf(c) (Eq. 7 of the paper).
    """
    f = lambda p: scene_sdf(p, transform, scale)
    hmin = 2.0 / (1 << max_level)

    def split(c, side, lev):
        return np.abs(f(c)) <= 0.5 * math.sqrt(3.0) * side

    def payload(c, side, lev):
        s = f(c)
        a = np.abs(s)
        d = np.select([a >= 0.4, a >= 0.2, a >= 0.1, a >= 0.05, a >= 0.025, a >= hmin],
                      [1, 2, 3, 4, 5, 6], 7)
        d = d + (hessian_frobenius(f, c, hmin) > hess_threshold)
        d = np.minimum(d, 8)
        if n_layers != 8:
            d = np.maximum(1, np.ceil(d * n_layers / 8.0)).astype(np.int64)
        d = np.minimum(d, n_layers)
        if far_field:
            near = a <= 0.5 * math.sqrt(3.0) * side
            d = np.where(near, d, 0)
        return d.astype(np.uint8), s.astype(np.float32)
    return build_octree(max_level, n_layers, split, payload)


def rotation(axis, angle: float) -> np.ndarray:
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


# --------------------------------------------------------------------------
# Query points
# --------------------------------------------------------------------------
def lattice(n: int) -> np.ndarray:
    """Marching-cubes lattice x_i = -1 + 2 i / (n - 1), computed in float64 and
    rounded to float32 once; points ordered with x fastest, then y, then z.
    Returns float32 [n^3, 3]."""
    t = (-1.0 + 2.0 * np.arange(n, dtype=np.float64) / (n - 1)).astype(np.float32)
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return np.ascontiguousarray(np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1))


def lattice_points(n: int, idx: np.ndarray) -> np.ndarray:
    """Lattice points at flat indices idx (same values as lattice(n)[idx])."""
    t = (-1.0 + 2.0 * np.arange(n, dtype=np.float64) / (n - 1)).astype(np.float32)
    idx = np.asarray(idx, np.int64)
    return np.ascontiguousarray(np.stack([t[idx % n], t[(idx // n) % n], t[idx // (n * n)]], axis=1))


def uniform_points(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    return g.uniform(lo, hi, (n, 3)).astype(np.float32)


def sample_indices(total: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices of range(total), sorted, from PCG64(seed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    if k >= total:
        return np.arange(total, dtype=np.int64)
    return np.sort(g.choice(total, size=k, replace=False)).astype(np.int64)


def boundary_points(level: int) -> np.ndarray:
    """Points on and one float32 ulp either side of every cell boundary of a
    2^level grid over [-1, 1], along each axis, with the other two
    coordinates at cell centres; plus the domain faces, points outside the
    domain and signed zeros.  float32 [k, 3]."""
    R = 1 << level
    b = (-1.0 + 2.0 * np.arange(R + 1) / R).astype(np.float32)
    vals = np.concatenate([b, np.nextafter(b, np.float32(-np.inf)), np.nextafter(b, np.float32(np.inf)),
                           np.array([-0.0, 0.0, -1.5, 1.5, -3e38, 3e38, np.inf, -np.inf], np.float32)])
    centres = (-1.0 + 2.0 * (np.arange(R) + 0.5) / R).astype(np.float32)
    g = np.random.Generator(np.random.PCG64(1234))
    pts = []
    for axis in range(3):
        for v in vals:
            o = g.choice(centres, size=2)
            p = [0, 0, 0]
            p[axis] = v
            p[(axis + 1) % 3] = o[0]
            p[(axis + 2) % 3] = o[1]
            pts.append(p)
    return np.array(pts, np.float32)


def pinhole_rays(width: int, height: int, fov_y_deg: float = 45.0, radius: float = 2.5,
                 azimuth_deg: float = 30.0, elevation_deg: float = 20.0):
    """Camera on a sphere of `radius` at (azimuth, elevation), looking at the
    origin with +y up.  Returns (origin float32[3], directions float32[h*w, 3])
    for pixel centres, row-major from the top-left."""
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    eye = radius * np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0]); right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    tan = math.tan(math.radians(fov_y_deg) / 2)
    aspect = width / height
    px = (np.arange(width) + 0.5) / width * 2 - 1
    py = 1 - (np.arange(height) + 0.5) / height * 2
    X, Y = np.meshgrid(px * tan * aspect, py * tan)
    d = fwd[None, :] + X.reshape(-1, 1) * right[None, :] + Y.reshape(-1, 1) * up[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return eye.astype(np.float32), d.astype(np.float32)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
def scene_surface_points(n: int, seed: int) -> np.ndarray:
    """n points on the zero level set of scene_sdf: points drawn uniformly on each primitive's
    surface (sphere: normalised Gaussian directions; torus: uniform angles, accepted with the
    area weight (R + r cos v) / (R + r)), kept where no other primitive contains them, float64."""
    g = np.random.Generator(np.random.PCG64(seed))
    spheres = [((-0.35, 0.0, 0.0), 0.30), ((0.35, 0.10, 0.0), 0.25), ((0.0, -0.30, 0.30), 0.20)]
    tc, R, r = np.array((0.0, 0.35, -0.20)), 0.35, 0.08
    out = []
    have = 0
    while have < n:
        k = max(4 * (n - have), 1024)
        parts = []
        for c, rad in spheres:
            v = g.standard_normal((k, 3))
            parts.append(np.asarray(c) + rad * v / np.linalg.norm(v, axis=1, keepdims=True))
        u, w = g.uniform(0, 2 * np.pi, k), g.uniform(0, 2 * np.pi, k)
        keep = g.uniform(0, 1, k) < (R + r * np.cos(w)) / (R + r)
        ring = R + r * np.cos(w)
        tor = np.stack([ring * np.cos(u), r * np.sin(w), ring * np.sin(u)], axis=1) + tc
        parts.append(tor[keep])
        p = np.concatenate(parts)
        p = p[np.abs(scene_sdf(p)) < 1e-9]
        p = p[g.permutation(len(p))]
        out.append(p)
        have += len(p)
    return np.concatenate(out)[:n]


def training_batch(n: int, seed: int, surface_frac: float = 0.6, sigma: float = 0.01):
    """A training batch as Sec. 4.1 samples it, on the analytic scene: surface_frac of the points
    on the surface, the rest surface points moved by Gaussian noise (sigma), all in [-1, 1]^3, and
    their exact SDF values as targets.  Returns (points float32 [n, 3], targets float32 [n])."""
    g = np.random.Generator(np.random.PCG64(seed))
    k = int(round(surface_frac * n))
    surf = scene_surface_points(n, seed + 1)
    jit = surf[k:] + sigma * g.standard_normal((n - k, 3))
    pts = np.clip(np.concatenate([surf[:k], jit]), -1.0, 1.0).astype(np.float32)
    pts = pts[g.permutation(n)]
    return pts, scene_sdf(pts.astype(np.float64)).astype(np.float32)


def serve_specs():
    """The three resident models of the serving workload, each with its own level-7 octree of
    the analytic scene (rotated and scaled per model): 8 x 256 SIREN (seed 1), 8 x 336 SIREN
    (seed 2), 6 x 128 ReLU on 64 Fourier features (sigma 10, seed 3)."""
    return [(siren_tmlp(8, 256, seed=1), scene_octree(7, 8)),
            (siren_tmlp(8, 336, seed=2), scene_octree(7, 8, transform=rotation([0, 1, 0], 0.5), scale=0.95)),
            (relu_ff_tmlp(6, 128, n_freq=64, sigma=10.0, seed=3),
             scene_octree(7, 6, transform=rotation([1, 1, 0], 0.7), scale=0.9))]


def config_tiny():
    """4 x 64 SIREN (seed 0), 8^3 voxel sphere map, 32^3 lattice."""
    return siren_tmlp(4, 64, seed=0), voxel_sphere_octree(3, 0.5), lattice(32)


def config_sand_siren(tail_kind: int = TAIL_LINEAR, far_field: bool = False, grid: int = 256):
    """8 x 256 SIREN (seed 1), level-7 scene octree, grid^3 lattice."""
    return siren_tmlp(8, 256, seed=1, tail_kind=tail_kind), scene_octree(7, 8, far_field), grid
